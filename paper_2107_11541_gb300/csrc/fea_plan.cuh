// fea_plan.cuh -- schedules for the row-owned (deterministic, atomic-free)
// assembly kernels, built once per pattern.
#pragma once
#include "fea_internal.cuh"

namespace fea {

// Builds the plan for this mesh; *out may be set to null when no row-owned
// kernel exists for the mesh (the atomic path is then used).
fea_status plan_build(fea_mesh* m, fea_pattern* p, fea_rowowned_plan** out);
void plan_destroy(fea_rowowned_plan* plan);
// True when plan_assemble can serve this call.
bool plan_supports(const fea_rowowned_plan* plan, int n_eq, int accumulate);
fea_status plan_assemble(const fea_rowowned_plan* plan, const AsmArgs<float>& a, cudaStream_t s);

}  // namespace fea
