// fea_plan.cuh -- schedules for the row-owned (deterministic, atomic-free in
// global memory) assembly kernel, built once per pattern and equation count.
#pragma once
#include "fea_internal.cuh"

namespace fea {

// Creates the (lazy) plan object of a pattern; *out is null when no row-owned
// kernel exists for the element type.
fea_status plan_build(fea_mesh* m, fea_pattern* p, fea_rowowned_plan** out);
void plan_destroy(fea_rowowned_plan* plan);
// Builds, on first use, the schedule for n_eq equations and batches of `batch` elements (0: the
// kernel's rule).  *ok is false when the row-owned kernel cannot serve this call (the atomic
// path is used instead).
fea_status plan_prepare(fea_rowowned_plan* plan, int n_eq, int batch, bool* ok);
// Equations a.eq0 .. a.eq0 + a.eq_count - 1 in `groups` groups of plan_group_size(eq_count, groups)
// (the last one smaller), batches of a.batch elements; plan_prepare must have succeeded for
// that group size and batch.
fea_status plan_assemble(fea_rowowned_plan* plan, const AsmArgs<float>& a, int accumulate, int groups, cudaStream_t s);
// The schedule key of a group size and batch (plan_trim keeps schedules by key).
int plan_key(int n_eq, int batch);
int plan_group_size(int n_eq, int groups);
// Element-parallel FP32 Hex8 (no schedule): atomics, the gather scratch (a.em) or the
// matrix-free residual (a.resid), for the launch's equations.
fea_status plan_elem(fea_rowowned_plan* plan, const AsmArgs<float>& a, cudaStream_t s);
// The same kernel with the node-major field scratch held by the caller (grown on demand):
// the Hex8 block of a mixed mesh, which has no plan.
fea_status hex8_elem(float*& fnode, size_t& fnode_bytes, const AsmArgs<float>& a, cudaStream_t s);
// Frees the schedules whose plan_key is not listed in keep.
void plan_trim(fea_rowowned_plan* plan, const std::vector<int>& keep);

}  // namespace fea
