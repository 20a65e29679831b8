// Persistent Jacobi-PCG for the coarse Poisson solves of CGP (Eqs. 12, 15),
// and the standalone CSR SpMV y = K x.
//
// One cooperative launch runs a whole solve.  The rows of an instance are
// split into contiguous chunks, one per block of the instance's block group;
// x, r, z and q of a row are only ever touched by the block that owns it, and
// only p (and x, during set-up and refinement) is read across blocks by the
// SpMV.  A CG iteration (Saad, Alg. 9.1) takes three group barriers:
//
//   A: beta = (r,z)/(r,z)_old, p = z + beta p           -> barrier (p complete)
//   B: q = K p, partial (p,q)                          -> barrier
//   C: alpha = (r,z)/(p,q); x += alpha p; r -= alpha q;
//      z = D^-1 r; partial (r,z), (r,r)                -> barrier
//
// Partial sums go to a per-block slot; after a barrier every block sums the
// slots in the same fixed order, so all blocks hold bit-identical scalars and
// the result is deterministic run to run.  Slots alternate between two banks
// so the next reduction never overwrites a slot still being read.
//
// The Neumann null space (constants) is handled by mean-zero projection of
// b, of x0 and of the final x.  MIXED precision wraps FP32 inner solves in
// FP64 iterative refinement: r = b - K x, r -= mean(r), stop test, inner
// PCG32 on K32 d = r32 to inner_tol, x += d, x -= mean(x).
//
// Barriers spin on a counter with a wall-clock limit; a block that gives up
// raises a flag that makes every other block leave at its next barrier, and
// the host reports CGP_ERR_TIMEOUT.  Blocks are grouped per instance so a
// batched launch can run independent systems side by side.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "cgp_internal.h"

namespace cgp {
namespace {

constexpr int NCOMP = 4;         // partial-sum components per reduction
constexpr int MAX_BLOCK = 1024;

struct Desc {
  int n;
  const int* rowptr;
  const int* col;
  const double* val;
  const float* val32;
  const double* dinv;
  const float* dinv32;
  const double* b;
  double* x;
  double* bp;
  double* r;
  double* z;
  double* p;
  double* q;
  float* r32;
  float* z32;
  float* p32;
  float* q32;
  float* d32;
  double* part;
  int part_stride;
  unsigned* bar;
  SolveResult* res;
  cgp_solve_info* out;  // optional device copy of the outcome
  int blk0, nblk;
  double tol, inner_tol;
  int max_it, max_sweeps, use_x0, mixed;
  long long spin_ns;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Shared {
  double red[NCOMP * 32];
  double tot[NCOMP];
  int flag;
};

// Barrier over the blocks of one instance.
struct Group {
  unsigned* bar;
  int* timeout;
  unsigned nblk;
  unsigned epoch;
  long long spin_ns;

  __device__ bool sync(Shared& sh) {
    __syncthreads();
    if (nblk == 1) return true;
    ++epoch;
    if (threadIdx.x == 0) {
      int ok = 1;
      __threadfence();
      atomicAdd(bar, 1u);
      const unsigned target = epoch * nblk;
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire(bar) < target) {
        if (*(volatile int*)timeout) { ok = 0; break; }
        if ((++spins & 31u) == 0 && (long long)(global_ns() - t0) > spin_ns) {
          atomicExch(timeout, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
      __threadfence();
      sh.flag = ok;
    }
    __syncthreads();
    return sh.flag != 0;
  }
};

// Sum NC per-thread values over the block; thread 0 stores them as this
// block's partials in bank (red & 1).
template <int NC>
__device__ __forceinline__ void put_partials(const Desc& d, int lb, int red, double (&v)[NC], Shared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double s = warp_sum(v[c]);
    if (lane == 0) sh.red[c * 32 + warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double s = lane < nw ? sh.red[c * 32 + lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) d.part[((red & 1) * NCOMP + c) * d.part_stride + lb] = s;
    }
  }
}

// After a barrier: totals of reduction `red`, identical in every block.
template <int NC>
__device__ __forceinline__ void get_totals(const Desc& d, int red, Shared& sh) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double* src = d.part + ((red & 1) * NCOMP + c) * d.part_stride;
      double s = 0.0;
      for (int j = lane; j < d.nblk; j += 32) s += __ldcg(src + j);
      s = warp_sum(s);
      if (lane == 0) sh.tot[c] = s;
    }
  }
  __syncthreads();
}

// Row-wise SpMV over rows [r0, r1) with T lanes per row; `op(i, s)` is called
// by lane 0 of the row's group with s = (A x)_i.  x is read through L2 (it is
// written by other blocks between barriers).
template <int T, typename V, typename Op>
__device__ __forceinline__ void spmv_rows(const int* __restrict__ rowptr, const int* __restrict__ col,
                                          const V* __restrict__ val, const V* x, int r0, int r1, Op op) {
  const int g = threadIdx.x / T, l = threadIdx.x % T, ng = blockDim.x / T;
  for (int base = r0; base < r1; base += ng) {
    const int i = base + g;
    V s = V(0);
    if (i < r1) {
      const int k1 = rowptr[i + 1];
      for (int k = rowptr[i] + l; k < k1; k += T) s = fma(val[k], __ldcg(x + col[k]), s);
    }
    if (T > 1) {
#pragma unroll
      for (int o = T / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, T);
    }
    if (i < r1 && l == 0) op(i, s);
  }
}

__device__ void finish(const Desc& d, int lb, int status, int its, int sweeps, double rel_rec, double rel_true,
                       double bnorm) {
  if (lb == 0 && threadIdx.x == 0) {
    d.res->status = status;
    d.res->iterations = its;
    d.res->sweeps = sweeps;
    d.res->rel_rec = rel_rec;
    d.res->rel_true = rel_true;
    d.res->bnorm = bnorm;
    if (d.out) {
      d.out->iterations = its;
      d.out->outer_sweeps = sweeps;
      d.out->rel_res_recursive = rel_rec;
      d.out->rel_res_true = rel_true;
      d.out->status = status;
    }
  }
}

// Block 0 marks the optional outcome record as timed out before any barrier;
// finish() overwrites it, so a record still saying TIMEOUT means some barrier
// of the solve gave up.
__device__ __forceinline__ void mark_pending(const Desc& d, int lb) {
  if (lb == 0 && threadIdx.x == 0 && d.out) {
    d.out->iterations = 0;
    d.out->outer_sweeps = 0;
    d.out->rel_res_recursive = 0.0;
    d.out->rel_res_true = 0.0;
    d.out->status = CGP_ERR_TIMEOUT;
  }
}

// Set-up shared by both precisions: bp = b - mean(b), x = x0 - mean(x0) or 0.
// Returns ||bp|| (identical in all blocks), or a negative value if the group
// barrier failed.
__device__ double setup(const Desc& d, int lb, int r0, int r1, Group& grp, Shared& sh, int& red) {
  const int tid = threadIdx.x, bd = blockDim.x;
  double v2[2] = {0.0, 0.0};
  for (int i = r0 + tid; i < r1; i += bd) {
    v2[0] += d.b[i];
    if (d.use_x0) v2[1] += d.x[i];
  }
  put_partials<2>(d, lb, red, v2, sh);
  if (!grp.sync(sh)) return -1.0;
  get_totals<2>(d, red, sh);
  ++red;
  const double mb = sh.tot[0] / d.n, mx = sh.tot[1] / d.n;
  double v1[1] = {0.0};
  for (int i = r0 + tid; i < r1; i += bd) {
    const double bi = d.b[i] - mb;
    d.bp[i] = bi;
    v1[0] += bi * bi;
    d.x[i] = d.use_x0 ? d.x[i] - mx : 0.0;
  }
  put_partials<1>(d, lb, red, v1, sh);
  if (!grp.sync(sh)) return -1.0;
  get_totals<1>(d, red, sh);
  ++red;
  return sqrt(sh.tot[0]);
}

// x -= mean(x) over the group, leaving x complete after a barrier.
__device__ bool project_x(const Desc& d, int lb, int r0, int r1, Group& grp, Shared& sh, int& red) {
  const int tid = threadIdx.x, bd = blockDim.x;
  double v1[1] = {0.0};
  for (int i = r0 + tid; i < r1; i += bd) v1[0] += d.x[i];
  put_partials<1>(d, lb, red, v1, sh);
  if (!grp.sync(sh)) return false;
  get_totals<1>(d, red, sh);
  ++red;
  const double mx = sh.tot[0] / d.n;
  for (int i = r0 + tid; i < r1; i += bd) d.x[i] -= mx;
  return grp.sync(sh);
}

// ||bp - K x||^2 over the group (x complete).
template <int T>
__device__ bool true_residual(const Desc& d, int lb, int r0, int r1, Group& grp, Shared& sh, int& red,
                              double& out) {
  double v1[1] = {0.0};
  spmv_rows<T, double>(d.rowptr, d.col, d.val, d.x, r0, r1, [&](int i, double s) {
    const double t = d.bp[i] - s;
    v1[0] += t * t;
  });
  put_partials<1>(d, lb, red, v1, sh);
  if (!grp.sync(sh)) return false;
  get_totals<1>(d, red, sh);
  ++red;
  out = sh.tot[0];
  return true;
}

template <int T>
__device__ void solve_fp64(const Desc& d, int lb) {
  __shared__ Shared sh;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int chunk = (d.n + d.nblk - 1) / d.nblk;
  const int r0 = min(d.n, lb * chunk), r1 = min(d.n, r0 + chunk);
  Group grp{d.bar, &d.res->timeout, (unsigned)d.nblk, 0u, d.spin_ns};
  int red = 0;

  const double bnorm = setup(d, lb, r0, r1, grp, sh, red);
  if (bnorm < 0.0) return;
  if (!isfinite(bnorm)) { finish(d, lb, CGP_ERR_NONFINITE, 0, 0, 0.0, 0.0, bnorm); return; }
  if (bnorm == 0.0) {
    for (int i = r0 + tid; i < r1; i += bd) d.x[i] = 0.0;
    finish(d, lb, CGP_OK, 0, 0, 0.0, 0.0, 0.0);
    return;
  }
  // r = bp - K x, z = D^-1 r, p = z
  {
    double v2[2] = {0.0, 0.0};
    spmv_rows<T, double>(d.rowptr, d.col, d.val, d.x, r0, r1, [&](int i, double s) {
      const double ri = d.bp[i] - s;
      const double zi = d.dinv[i] * ri;
      d.r[i] = ri;
      d.z[i] = zi;
      d.p[i] = zi;
      v2[0] += ri * zi;
      v2[1] += ri * ri;
    });
    put_partials<2>(d, lb, red, v2, sh);
    if (!grp.sync(sh)) return;
  }
  int k = 0, status = CGP_ERR_NOT_CONVERGED;
  double rz_old = 0.0, rnorm = 0.0;
  const double stop = d.tol * bnorm;
  while (true) {
    get_totals<2>(d, red, sh);
    ++red;
    const double rz = sh.tot[0];
    rnorm = sqrt(sh.tot[1]);
    if (!isfinite(rnorm)) { status = CGP_ERR_NONFINITE; break; }
    if (rnorm <= stop) { status = CGP_OK; break; }
    if (k >= d.max_it) { status = CGP_ERR_NOT_CONVERGED; break; }
    if (k > 0) {  // phase A
      const double beta = rz / rz_old;
      for (int i = r0 + tid; i < r1; i += bd) d.p[i] = fma(beta, d.p[i], d.z[i]);
      if (!grp.sync(sh)) return;
    }
    rz_old = rz;
    {  // phase B
      double v1[1] = {0.0};
      spmv_rows<T, double>(d.rowptr, d.col, d.val, d.p, r0, r1, [&](int i, double s) {
        d.q[i] = s;
        v1[0] += d.p[i] * s;
      });
      put_partials<1>(d, lb, red, v1, sh);
      if (!grp.sync(sh)) return;
      get_totals<1>(d, red, sh);
      ++red;
    }
    const double pq = sh.tot[0];
    if (!(pq > 0.0)) { status = isfinite(pq) ? CGP_ERR_BREAKDOWN : CGP_ERR_NONFINITE; break; }
    const double alpha = rz / pq;
    {  // phase C
      double v2[2] = {0.0, 0.0};
      for (int i = r0 + tid; i < r1; i += bd) {
        const double pi = d.p[i];
        d.x[i] = fma(alpha, pi, d.x[i]);
        const double ri = fma(-alpha, d.q[i], d.r[i]);
        const double zi = d.dinv[i] * ri;
        d.r[i] = ri;
        d.z[i] = zi;
        v2[0] += ri * zi;
        v2[1] += ri * ri;
      }
      put_partials<2>(d, lb, red, v2, sh);
      if (!grp.sync(sh)) return;
    }
    ++k;
  }
  if (!project_x(d, lb, r0, r1, grp, sh, red)) return;
  double tr = 0.0;
  if (!true_residual<T>(d, lb, r0, r1, grp, sh, red, tr)) return;
  finish(d, lb, status, k, 0, rnorm / bnorm, sqrt(tr) / bnorm, bnorm);
}

template <int T>
__device__ void solve_mixed(const Desc& d, int lb) {
  __shared__ Shared sh;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int chunk = (d.n + d.nblk - 1) / d.nblk;
  const int r0 = min(d.n, lb * chunk), r1 = min(d.n, r0 + chunk);
  Group grp{d.bar, &d.res->timeout, (unsigned)d.nblk, 0u, d.spin_ns};
  int red = 0;

  const double bnorm = setup(d, lb, r0, r1, grp, sh, red);
  if (bnorm < 0.0) return;
  if (!isfinite(bnorm)) { finish(d, lb, CGP_ERR_NONFINITE, 0, 0, 0.0, 0.0, bnorm); return; }
  if (bnorm == 0.0) {
    for (int i = r0 + tid; i < r1; i += bd) d.x[i] = 0.0;
    finish(d, lb, CGP_OK, 0, 0, 0.0, 0.0, 0.0);
    return;
  }
  int total = 0, sweeps = 0, status = CGP_ERR_NOT_CONVERGED;
  double rel = 0.0;
  while (true) {
    // ---- FP64 residual r = bp - K x and its projection ----
    {
      double v1[1] = {0.0};
      spmv_rows<T, double>(d.rowptr, d.col, d.val, d.x, r0, r1, [&](int i, double s) {
        const double ri = d.bp[i] - s;
        d.r[i] = ri;
        v1[0] += ri;
      });
      put_partials<1>(d, lb, red, v1, sh);
      if (!grp.sync(sh)) return;
      get_totals<1>(d, red, sh);
      ++red;
    }
    const double mr = sh.tot[0] / d.n;
    {
      double v1[1] = {0.0};
      for (int i = r0 + tid; i < r1; i += bd) {
        const double ri = d.r[i] - mr;
        v1[0] += ri * ri;
        d.r32[i] = (float)ri;
      }
      put_partials<1>(d, lb, red, v1, sh);
      if (!grp.sync(sh)) return;
      get_totals<1>(d, red, sh);
      ++red;
    }
    rel = sqrt(sh.tot[0]) / bnorm;
    if (!isfinite(rel)) { status = CGP_ERR_NONFINITE; break; }
    if (rel <= d.tol) { status = CGP_OK; break; }
    if (sweeps >= d.max_sweeps || total >= d.max_it) { status = CGP_ERR_NOT_CONVERGED; break; }

    // ---- FP32 inner PCG: K32 e = r32 from e = 0 ----
    {
      double v2[2] = {0.0, 0.0};
      for (int i = r0 + tid; i < r1; i += bd) {
        const float ri = d.r32[i];
        const float zi = d.dinv32[i] * ri;
        d.z32[i] = zi;
        d.p32[i] = zi;
        d.d32[i] = 0.0f;
        v2[0] += (double)(ri * zi);
        v2[1] += (double)(ri * ri);
      }
      put_partials<2>(d, lb, red, v2, sh);
      if (!grp.sync(sh)) return;
    }
    int k = 0;
    float rz_old = 0.0f;
    float r0n = -1.0f;
    bool inner_bad = false, capped = false;
    while (true) {
      get_totals<2>(d, red, sh);
      ++red;
      const float rz = (float)sh.tot[0];
      const float rn = sqrtf((float)sh.tot[1]);
      if (r0n < 0.0f) r0n = rn;
      if (!isfinite(rn)) { inner_bad = true; break; }
      if (rn <= (float)d.inner_tol * r0n) break;
      if (total + k >= d.max_it) { capped = true; break; }
      if (k > 0) {
        const float beta = rz / rz_old;
        for (int i = r0 + tid; i < r1; i += bd) d.p32[i] = fmaf(beta, d.p32[i], d.z32[i]);
        if (!grp.sync(sh)) return;
      }
      rz_old = rz;
      {
        double v1[1] = {0.0};
        float acc = 0.0f;
        spmv_rows<T, float>(d.rowptr, d.col, d.val32, d.p32, r0, r1, [&](int i, float s) {
          d.q32[i] = s;
          acc = fmaf(d.p32[i], s, acc);
        });
        v1[0] = acc;
        put_partials<1>(d, lb, red, v1, sh);
        if (!grp.sync(sh)) return;
        get_totals<1>(d, red, sh);
        ++red;
      }
      const float pq = (float)sh.tot[0];
      if (!(pq > 0.0f)) { inner_bad = !isfinite(pq); break; }
      const float alpha = rz / pq;
      {
        float a0 = 0.0f, a1 = 0.0f;
        for (int i = r0 + tid; i < r1; i += bd) {
          const float pi = d.p32[i];
          d.d32[i] = fmaf(alpha, pi, d.d32[i]);
          const float ri = fmaf(-alpha, d.q32[i], d.r32[i]);
          const float zi = d.dinv32[i] * ri;
          d.r32[i] = ri;
          d.z32[i] = zi;
          a0 = fmaf(ri, zi, a0);
          a1 = fmaf(ri, ri, a1);
        }
        double v2[2] = {(double)a0, (double)a1};
        put_partials<2>(d, lb, red, v2, sh);
        if (!grp.sync(sh)) return;
      }
      ++k;
    }
    total += k;
    if (inner_bad) { status = CGP_ERR_NONFINITE; break; }
    // ---- FP64 correction and projection ----
    for (int i = r0 + tid; i < r1; i += bd) d.x[i] += (double)d.d32[i];
    if (!project_x(d, lb, r0, r1, grp, sh, red)) return;
    ++sweeps;
    if (k == 0 && !capped) { status = CGP_ERR_BREAKDOWN; break; }  // the inner solve made no progress
  }
  finish(d, lb, status, total, sweeps, rel, rel, bnorm);
}

template <int T>
__global__ void __launch_bounds__(MAX_BLOCK) pcg_persistent_kernel(Desc d) {
  mark_pending(d, blockIdx.x);
  if (d.mixed)
    solve_mixed<T>(d, blockIdx.x);
  else
    solve_fp64<T>(d, blockIdx.x);
}

// ---------------------------------------------------------------------------
// standalone SpMV: T lanes per row, grid-stride over row groups
// ---------------------------------------------------------------------------
template <int T, typename V>
__global__ void __launch_bounds__(256) spmv_kernel(int n, const int* __restrict__ rowptr,
                                                   const int* __restrict__ col, const V* __restrict__ val,
                                                   const V* __restrict__ x, V* __restrict__ y) {
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) / T, l = threadIdx.x % T;
  const int ng = gridDim.x * blockDim.x / T;
  for (int base = 0; base < n; base += ng) {
    const int i = base + g;
    V s = V(0);
    if (i < n) {
      const int k1 = rowptr[i + 1];
      for (int k = rowptr[i] + l; k < k1; k += T) s = fma(val[k], __ldg(x + col[k]), s);
    }
    if (T > 1) {
#pragma unroll
      for (int o = T / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, T);
    }
    if (i < n && l == 0) y[i] = s;
  }
}

using PcgFn = void (*)(Desc);

PcgFn pcg_kernel_for(int lanes) {
  switch (lanes) {
    case 1: return pcg_persistent_kernel<1>;
    case 2: return pcg_persistent_kernel<2>;
    case 4: return pcg_persistent_kernel<4>;
    case 8: return pcg_persistent_kernel<8>;
    case 32: return pcg_persistent_kernel<32>;
    default: return nullptr;
  }
}

struct DevInfo {
  int sms = 0;
};

DevInfo dev_info(int device) {
  static std::mutex mu;
  static DevInfo cache[64];
  std::lock_guard<std::mutex> lk(mu);
  if (device < 0 || device >= 64) return DevInfo{};
  if (cache[device].sms == 0) cudaDeviceGetAttribute(&cache[device].sms, cudaDevAttrMultiProcessorCount, device);
  return cache[device];
}

int coresident_blocks(PcgFn fn, int block, int device) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, block, 0) != cudaSuccess) return 0;
  return per_sm * dev_info(device).sms;
}

}  // namespace

int solver_max_blocks(int device) {
  int sms = dev_info(device).sms;
  if (sms <= 0) sms = 160;
  return sms * 32;  // upper bound on co-resident blocks of >= 64 threads
}

int launch_solve(cgp_mesh_impl* m, const double* b, double* x, const cgp_solve_opts& o, cgp_solve_info* info_dev,
                 cudaStream_t s) {
  const bool mixed = o.precision == CGP_MIXED;
  const SolverTuning& tu = m->tune[mixed ? CGP_TUNE_SOLVE_MIXED : CGP_TUNE_SOLVE_FP64];
  const int lanes = tu.lanes > 0 ? tu.lanes : 1;
  const int block = tu.block > 0 ? tu.block : 512;
  PcgFn fn = pcg_kernel_for(lanes);
  if (!fn) return fail(CGP_ERR_INVALID_ARG, "solver tuning: lanes must be 1, 2, 4, 8 or 32");
  if (block < 64 || block > MAX_BLOCK || block % 32 != 0 || block % lanes != 0)
    return fail(CGP_ERR_INVALID_ARG, "solver tuning: block must be a multiple of 32 in [64, 1024]");
  const int cap = std::min(coresident_blocks(fn, block, m->device), m->max_blocks);
  if (cap <= 0) return fail(CGP_ERR_CUDA, "solver: kernel cannot be resident on this device");
  int nblk = tu.blocks;
  if (nblk <= 0) nblk = m->n_c <= 16384 ? 1 : (m->n_c + block - 1) / block;
  nblk = std::max(1, std::min(nblk, std::min(cap, m->n_c)));
  // barrier epochs stay far below 2^32 / nblk
  const long long max_epochs = 8LL + 4LL * (long long)std::max(o.max_it, 1) + 8LL * std::max(o.max_sweeps, 1);
  if (max_epochs * nblk >= (1LL << 31)) return fail(CGP_ERR_INVALID_ARG, "solver: max_it too large");

  Desc d{};
  d.n = m->n_c;
  d.rowptr = m->rowptr;
  d.col = m->col;
  d.val = m->K;
  d.val32 = m->K32;
  d.dinv = m->dinv;
  d.dinv32 = m->dinv32;
  d.b = b;
  d.x = x;
  d.bp = m->bp;
  d.r = m->r;
  d.z = m->z;
  d.p = m->p;
  d.q = m->q;
  d.r32 = m->r32;
  d.z32 = m->z32;
  d.p32 = m->p32;
  d.q32 = m->q32;
  d.d32 = m->d32;
  d.part = m->part;
  d.part_stride = m->max_blocks;
  d.bar = m->bar;
  d.res = m->res;
  d.out = info_dev;
  d.blk0 = 0;
  d.nblk = nblk;
  d.tol = o.tol;
  d.inner_tol = o.inner_tol;
  d.max_it = o.max_it;
  d.max_sweeps = o.max_sweeps;
  d.use_x0 = o.use_x0;
  d.mixed = mixed ? 1 : 0;
  d.spin_ns = 2000000000LL;

  CGP_CUDA(cudaMemsetAsync(m->bar, 0, 64, s));
  CGP_CUDA(cudaMemsetAsync(m->res, 0, sizeof(SolveResult), s));
  void* args[] = {&d};
  CGP_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3(nblk), dim3(block), args, 0, s));
  return CGP_OK;
}

using SpmvFn64 = void (*)(int, const int*, const int*, const double*, const double*, double*);
using SpmvFn32 = void (*)(int, const int*, const int*, const float*, const float*, float*);

template <typename V>
void (*spmv_for(int lanes))(int, const int*, const int*, const V*, const V*, V*) {
  switch (lanes) {
    case 1: return spmv_kernel<1, V>;
    case 2: return spmv_kernel<2, V>;
    case 4: return spmv_kernel<4, V>;
    case 8: return spmv_kernel<8, V>;
    case 32: return spmv_kernel<32, V>;
    default: return nullptr;
  }
}

int launch_solve_fp64_raw(int device, const RawSystem& sys, const RawScratch& scr, const double* b, double* x,
                          const cgp_solve_opts& o, cudaStream_t s) {
  const int block = 512;
  PcgFn fn = pcg_kernel_for(1);
  const int cap = std::min(coresident_blocks(fn, block, device), scr.max_blocks);
  if (cap <= 0) return fail(CGP_ERR_CUDA, "solver: kernel cannot be resident on this device");
  int nblk = sys.n <= 16384 ? 1 : (sys.n + block - 1) / block;
  nblk = std::max(1, std::min(nblk, std::min(cap, sys.n)));
  const long long max_epochs = 8LL + 4LL * (long long)std::max(o.max_it, 1);
  if (max_epochs * nblk >= (1LL << 31)) return fail(CGP_ERR_INVALID_ARG, "solver: max_it too large");
  Desc d{};
  d.n = sys.n;
  d.rowptr = sys.rowptr;
  d.col = sys.col;
  d.val = sys.val;
  d.dinv = sys.dinv;
  d.b = b;
  d.x = x;
  d.bp = scr.bp;
  d.r = scr.r;
  d.z = scr.z;
  d.p = scr.p;
  d.q = scr.q;
  d.part = scr.part;
  d.part_stride = scr.max_blocks;
  d.bar = scr.bar;
  d.res = scr.res;
  d.out = nullptr;
  d.blk0 = 0;
  d.nblk = nblk;
  d.tol = o.tol;
  d.inner_tol = o.inner_tol;
  d.max_it = o.max_it;
  d.max_sweeps = 1;
  d.use_x0 = o.use_x0;
  d.mixed = 0;
  d.spin_ns = 2000000000LL;
  void* args[] = {&d};
  CGP_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3(nblk), dim3(block), args, 0, s));
  return CGP_OK;
}

int launch_spmv(cgp_mesh_impl* m, int precision, const void* x, void* y, cudaStream_t s) {
  const int sms = std::max(1, dev_info(m->device).sms);
  const SolverTuning& tu = m->tune[precision == CGP_FP64 ? CGP_TUNE_SPMV_FP64 : CGP_TUNE_SPMV_FP32];
  const int block = tu.block > 0 ? tu.block : 256;
  const int lanes = tu.lanes > 0 ? tu.lanes : (precision == CGP_FP64 ? 1 : 4);
  long long grid = tu.blocks;
  if (grid <= 0) {
    grid = ((long long)m->n_c * lanes + block - 1) / block;
    grid = std::max(1LL, std::min(grid, (long long)sms * 16));
  }
  if (precision == CGP_FP64) {
    auto fn = spmv_for<double>(lanes);
    if (!fn) return fail(CGP_ERR_INVALID_ARG, "spmv tuning: bad lanes");
    fn<<<(int)grid, block, 0, s>>>(m->n_c, m->rowptr, m->col, m->K, (const double*)x, (double*)y);
  } else {
    auto fn = spmv_for<float>(lanes);
    if (!fn) return fail(CGP_ERR_INVALID_ARG, "spmv tuning: bad lanes");
    fn<<<(int)grid, block, 0, s>>>(m->n_c, m->rowptr, m->col, m->K32, (const float*)x, (float*)y);
  }
  CGP_CUDA(cudaGetLastError());
  return CGP_OK;
}

// ---------------------------------------------------------------------------
// barrier self-test: the last `absent` blocks never arrive
// ---------------------------------------------------------------------------
__global__ void barrier_selftest_kernel(unsigned* bar, int* timeout, int nblk, int absent, long long spin_ns,
                                        int* ok_count) {
  __shared__ Shared sh;
  if ((int)blockIdx.x >= nblk - absent) return;
  Group grp{bar, timeout, (unsigned)nblk, 0u, spin_ns};
  const bool ok = grp.sync(sh);
  if (threadIdx.x == 0 && ok) atomicAdd(ok_count, 1);
}

}  // namespace cgp

using namespace cgp;

static int check_solve_args(cgp_mesh m, const double* b, double* x, const cgp_solve_opts* opts, cgp_solve_opts& o) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_poisson_solve: NULL mesh");
  if (!b || !x) return fail(CGP_ERR_INVALID_ARG, "cgp_poisson_solve: NULL b or x");
  o = cgp_solve_opts{1e-8, 20000, CGP_FP64, 1e-4, 0, 50};
  if (opts) o = *opts;
  if (!(o.tol >= 0.0) || o.max_it < 0) return fail(CGP_ERR_INVALID_ARG, "cgp_poisson_solve: bad tol or max_it");
  if (o.precision != CGP_FP64 && o.precision != CGP_MIXED)
    return fail(CGP_ERR_INVALID_ARG, "cgp_poisson_solve: unknown precision");
  if (o.precision == CGP_MIXED && !(o.inner_tol > 0.0 && o.inner_tol < 1.0))
    return fail(CGP_ERR_INVALID_ARG, "cgp_poisson_solve: inner_tol must be in (0, 1)");
  if (o.max_sweeps <= 0) o.max_sweeps = 50;
  return CGP_OK;
}

extern "C" int cgp_poisson_solve_async(cgp_mesh m, const double* b, double* x, const cgp_solve_opts* opts,
                                       cgp_solve_info* info_dev, void* stream) {
  cgp_solve_opts o;
  int st = check_solve_args(m, b, x, opts, o);
  if (st != CGP_OK) return st;
  return launch_solve(m, b, x, o, info_dev, (cudaStream_t)stream);
}

extern "C" int cgp_poisson_solve(cgp_mesh m, const double* b, double* x, const cgp_solve_opts* opts,
                                 cgp_solve_info* info, void* stream) {
  cgp_solve_opts o;
  int st0 = check_solve_args(m, b, x, opts, o);
  if (st0 != CGP_OK) return st0;
  cudaStream_t s = (cudaStream_t)stream;
  int st = launch_solve(m, b, x, o, nullptr, s);
  if (st != CGP_OK) return st;
  if (!info) return CGP_OK;
  CGP_CUDA(cudaMemcpyAsync(m->h_res, m->res, sizeof(SolveResult), cudaMemcpyDeviceToHost, s));
  CGP_CUDA(cudaStreamSynchronize(s));
  const SolveResult& r = *m->h_res;
  info->iterations = r.iterations;
  info->outer_sweeps = r.sweeps;
  info->rel_res_recursive = r.rel_rec;
  info->rel_res_true = r.rel_true;
  info->status = r.timeout ? CGP_ERR_TIMEOUT : r.status;
  if (info->status == CGP_ERR_TIMEOUT) return fail(CGP_ERR_TIMEOUT, "cgp_poisson_solve: a grid barrier timed out");
  if (info->status != CGP_OK) {
    const char* what = info->status == CGP_ERR_NOT_CONVERGED ? "not converged"
                       : info->status == CGP_ERR_BREAKDOWN  ? "breakdown (p.Kp <= 0)"
                                                            : "non-finite value";
    return fail(info->status, std::string("cgp_poisson_solve: ") + what);
  }
  return CGP_OK;
}

static bool valid_shape(int block, int lanes) {
  if (block != 0 && (block < 64 || block > MAX_BLOCK || block % 32 != 0)) return false;
  if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 32) return false;
  return true;
}

extern "C" int cgp_set_tuning(cgp_mesh m, int what, int block, int lanes, int blocks) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_set_tuning: NULL mesh");
  if (what < 0 || what > 3) return fail(CGP_ERR_INVALID_ARG, "cgp_set_tuning: unknown target");
  if (!valid_shape(block, lanes) || blocks < 0)
    return fail(CGP_ERR_INVALID_ARG, "cgp_set_tuning: block must be 0 or a multiple of 32 in [64, 1024], "
                                     "lanes 0, 1, 2, 4, 8 or 32, blocks >= 0");
  m->tune[what] = SolverTuning{block, lanes, blocks};
  return CGP_OK;
}

extern "C" int cgp_get_tuning(cgp_mesh m, int what, int* block, int* lanes, int* blocks) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_get_tuning: NULL mesh");
  if (what < 0 || what > 3) return fail(CGP_ERR_INVALID_ARG, "cgp_get_tuning: unknown target");
  if (block) *block = m->tune[what].block;
  if (lanes) *lanes = m->tune[what].lanes;
  if (blocks) *blocks = m->tune[what].blocks;
  return CGP_OK;
}

extern "C" int cgp_barrier_selftest(int nblk, int absent, long long spin_ns, void* stream) {
  if (nblk < 1 || nblk > 1024 || absent < 0 || absent >= nblk || spin_ns <= 0)
    return fail(CGP_ERR_INVALID_ARG, "cgp_barrier_selftest: need 1 <= nblk <= 1024, 0 <= absent < nblk");
  cudaStream_t s = (cudaStream_t)stream;
  int device = 0;
  CGP_CUDA(cudaGetDevice(&device));
  int per_sm = 0;
  CGP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)barrier_selftest_kernel, 64, 0));
  if (per_sm * dev_info(device).sms < nblk)
    return fail(CGP_ERR_INVALID_ARG, "cgp_barrier_selftest: nblk exceeds the co-resident capacity");
  void* buf = nullptr;
  CGP_CUDA(cudaMalloc(&buf, 256));
  unsigned* bar = (unsigned*)buf;
  int* timeout = (int*)((char*)buf + 64);
  int* ok_count = (int*)((char*)buf + 128);
  int h[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(buf, 0, 256, s);
  if (e == cudaSuccess) {
    void* args[] = {&bar, &timeout, &nblk, &absent, &spin_ns, &ok_count};
    e = cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, dim3(nblk), dim3(64), args, 0, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h[0], timeout, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h[1], ok_count, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "cgp_barrier_selftest");
  if (h[0]) return fail(CGP_ERR_TIMEOUT, "cgp_barrier_selftest: barrier timed out (" + std::to_string(h[1]) +
                                             " blocks passed)");
  if (h[1] != nblk - absent) return fail(CGP_ERR_CUDA, "cgp_barrier_selftest: blocks missing without timeout");
  return CGP_OK;
}

extern "C" int cgp_spmv(cgp_mesh m, int precision, const void* x, void* y, void* stream) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_spmv: NULL mesh");
  if (!x || !y) return fail(CGP_ERR_INVALID_ARG, "cgp_spmv: NULL vector");
  if (precision != CGP_FP64 && precision != 1) return fail(CGP_ERR_INVALID_ARG, "cgp_spmv: unknown precision");
  return launch_spmv(m, precision, x, y, (cudaStream_t)stream);
}
