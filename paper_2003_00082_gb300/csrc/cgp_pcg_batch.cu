// Kernels of the batched persistent solver: many independent systems in one
// cooperative launch, each on its own group of blocks (the solve loops are
// those of the single-system kernel, cgp_solver.cuh).  Compiled as a unit of
// its own so that it builds in parallel with the rest of the solver.
#include "cgp_solver.cuh"

namespace cgp {
namespace {

// Many independent systems in one launch: block b runs instance
// blk_inst[b] as local block b - blk0 of that instance's group.
template <int T, bool RES>
__global__ void __launch_bounds__(MAX_BLOCK)
    pcg_batched_kernel(const Desc* __restrict__ descs, const int* __restrict__ blk_inst,
                       unsigned long long* t_start) {
  __shared__ Shared sh;
  if (t_start && blockIdx.x == 0 && threadIdx.x == 0) *t_start = global_ns();
  const Desc& d = descs[blk_inst[blockIdx.x]];
  const int lb = blockIdx.x - d.blk0;
  mark_pending(d, lb);
  if (d.mixed)
    solve_mixed<T, RES>(d, lb, sh);
  else if (d.classic)
    solve_fp64<T, RES>(d, lb, sh);
  else
    solve_fp64_sr<T, RES>(d, lb, sh);
}

}  // namespace

const void* batched_kernel_ptr(int lanes, bool res) {
  switch (lanes) {
    case 1: return res ? (const void*)pcg_batched_kernel<1, true> : (const void*)pcg_batched_kernel<1, false>;
    case 2: return res ? (const void*)pcg_batched_kernel<2, true> : (const void*)pcg_batched_kernel<2, false>;
    case 4: return res ? (const void*)pcg_batched_kernel<4, true> : (const void*)pcg_batched_kernel<4, false>;
    case 8: return res ? (const void*)pcg_batched_kernel<8, true> : (const void*)pcg_batched_kernel<8, false>;
    case 32: return res ? (const void*)pcg_batched_kernel<32, true> : (const void*)pcg_batched_kernel<32, false>;
    default: return nullptr;
  }
}

}  // namespace cgp
