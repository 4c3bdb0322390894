// fea_rowowned.cu -- row-owned assembly (placeholder: no schedule yet).
#include "fea_plan.cuh"

struct fea_rowowned_plan {
  int dummy;
};

namespace fea {

fea_status plan_build(fea_mesh*, fea_pattern*, fea_rowowned_plan** out) {
  *out = nullptr;
  return FEA_OK;
}
void plan_destroy(fea_rowowned_plan* plan) { delete plan; }
bool plan_supports(const fea_rowowned_plan* plan, int, int) { return plan != nullptr; }
fea_status plan_assemble(const fea_rowowned_plan*, const AsmArgs<float>&, cudaStream_t) {
  return fail(FEA_ERR_STATE, "row-owned plan unavailable");
}

}  // namespace fea
