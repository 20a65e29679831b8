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
// FP32 CG (single-reduction form) on K32 e = r to inner_tol, x += e,
// x -= mean(x).
//
// Barriers spin on a counter with a wall-clock limit; a block that gives up
// raises a flag that makes every other block leave at its next barrier, and
// the host reports CGP_ERR_TIMEOUT.  Blocks are grouped per instance so a
// batched launch can run independent systems side by side.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cgp_fixed.h"
#include "cgp_internal.h"
#include "cgp_sync.h"

namespace cgp {
namespace {

constexpr int NCOMP = 4;         // partial-sum components per reduction
constexpr int MAX_BLOCK = 512;   // threads per block of the persistent solver (<= 128 registers each)

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
  double* p2;         // second buffer of p (FP64 solver)
  double* q;
  double* pub64;      // FP64 single-reduction: published R[2], W[2], S[2] ([6][n])
  float* f32pub;      // mixed: published R[2], W[2], S[2] ([6][n])
  float* f32own;      // mixed without RES: own r, u, w, p, s, e ([6][n])
  float* fpart;       // mixed: FP32 partial slots [2][NCOMP][part_stride]
  double* part;
  unsigned long long* tpart;  // FP64 single-reduction: tagged slots [2][3][part_stride] (128-bit)
  int part_stride;
  unsigned* bar;
  SolveResult* res;
  cgp_solve_info* out;  // optional device copy of the outcome
  int blk0, nblk;
  double tol, inner_tol;
  int max_it, max_sweeps, use_x0, mixed;
  int classic;        // FP64: two barriers per iteration (Saad, Alg. 9.1) instead of the single-reduction form
  int tagged;         // FP64 single-reduction: reductions through tagged slots instead of the group barrier
  const unsigned char* fixed;  // far-field Dirichlet rows (phi = 0), or NULL for the natural condition everywhere
  int res_nnz_cap;    // RES: capacity of the shared-memory CSR slice
  int halo_cap;       // RES: capacity of the halo gather buffer
  const int* lcol;    // RES: columns renumbered per block (halo plan)
  const int* hptr;    // RES: halo list of each block
  const int* hidx;
  long long spin_ns;
};

// Rows held at zero by the far-field Dirichlet condition; with it, K has no
// null space and b, x0 and x are not projected to mean zero.
__device__ __forceinline__ bool is_fixed(const Desc& d, int i) { return d.fixed && d.fixed[i]; }

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Shared {
  unsigned long long wlo[3][32];  // per-warp fixed-point partials of one reduction
  long long whi[3][32];
  int wexp[3][32];
  double tot[NCOMP];
  double sc[8];                 // scalars computed by one lane and broadcast
  int isc[4];
  float fred[4][32];            // FP32 reductions of the inner solve
  float ftot[4];
  float fsc[8];
  int flag;
  int tflag;                    // outcome of the last tagged reduction's wait
};

// Barrier over the blocks of one instance (cgp_sync.h): a block that gives
// up makes every other block leave at its next barrier.
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
    if (threadIdx.x == 0) sh.flag = barrier_arrive_wait(bar, timeout, nblk, epoch, spin_ns) ? 1 : 0;
    __syncthreads();
    return sh.flag != 0;
  }

  // The same barrier split in two: work between arrive() and wait() overlaps
  // the other blocks' arrival; it must not write what other blocks read.
  __device__ void arrive() {
    __syncthreads();
    if (nblk == 1) return;
    ++epoch;
    if (threadIdx.x == 0) red_release_add(bar, 1u);
  }
  __device__ bool wait(Shared& sh) {
    if (nblk > 1 && threadIdx.x == 0) sh.flag = barrier_wait(bar, timeout, nblk, epoch, spin_ns) ? 1 : 0;
    __syncthreads();
    return nblk == 1 || sh.flag != 0;
  }
  // The wait of one thread (no block barrier): false when it gave up.
  __device__ bool wait_one() { return nblk == 1 || barrier_wait(bar, timeout, nblk, epoch, spin_ns); }
};

__device__ __forceinline__ fx::I128 shfl_xor_i128(fx::I128 a, int o) {
  const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)a, o);
  const long long hi = __shfl_xor_sync(0xffffffffu, (long long)(a >> 64), o);
  return ((fx::I128)hi << 64) | (fx::I128)lo;
}

__device__ __forceinline__ fx::I128 warp_sum_i128(fx::I128 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += shfl_xor_i128(a, o);
  return a;
}

// Warp-wide fixed-point sum of one double per lane: returns the warp's common
// exponent in E and the aligned integer sum (identical on every lane).
__device__ __forceinline__ fx::I128 warp_fx_sum(double v, int& E) {
  const int e = fx::exponent_of(v);
  E = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
  const fx::I128 x = E < fx::kBadExp ? fx::image(v, E) : (fx::I128)0;
  return warp_sum_i128(x);
}

// Partial-sum slot of (bank, component, block): {lo, hi, exponent} as 64-bit words.
__device__ __forceinline__ unsigned long long* part_slot(const Desc& d, int red, int c, int blk) {
  return reinterpret_cast<unsigned long long*>(d.part) + 4 * ((size_t)((red & 1) * NCOMP + c) * d.part_stride + blk);
}

// Tagged slots (cgp_fixed.h: fx::pack_tagged): one 128-bit word per (bank,
// component, block) that says by itself whether it holds reduction `red`, so
// a block can read the slots while it waits for the group barrier instead of
// after it.  A block zeroes its slots at the start of a launch.
__device__ __forceinline__ ulonglong2* tag_slot(const Desc& d, int red, int c, int blk) {
  return reinterpret_cast<ulonglong2*>(d.tpart) + ((size_t)((red & 1) * 3 + c) * d.part_stride + blk);
}

// Sum NC (<= 3) per-thread values over the block; warp c then folds
// component c over the warps and stores it as this block's partial in bank
// (red & 1): untagged in d.part, or TAGGED in d.tpart.  The sums are exact
// fixed-point integer sums (cgp_fixed.h): they run on the integer pipe, cost
// no FP64 instructions, and do not depend on the order of the terms.
template <int NC, bool TAGGED = false>
__device__ __forceinline__ void put_partials(const Desc& d, int lb, int red, double (&v)[NC], Shared& sh) {
  static_assert(NC >= 1 && NC <= 3, "one to three components per reduction");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    int E;
    const fx::I128 x = warp_fx_sum(v[c], E);
    if (lane == 0) {
      sh.wlo[c][warp] = (unsigned long long)x;
      sh.whi[c][warp] = (long long)(x >> 64);
      sh.wexp[c][warp] = E;
    }
  }
  if (TAGGED && threadIdx.x == 0) sh.tflag = 1;
  __syncthreads();
  for (int c = warp; c < NC; c += nw) {
    fx::I128 x = 0;
    int e = 1;
    if (lane < nw) {
      x = ((fx::I128)sh.whi[c][lane] << 64) | (fx::I128)sh.wlo[c][lane];
      e = sh.wexp[c][lane];
    }
    const int E = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
    x = warp_sum_i128(E < fx::kBadExp ? fx::sar(x, E - e) : (fx::I128)0);
    if (lane == 0) {
      if (TAGGED) {
        uint64_t lo, hi;
        fx::pack_tagged(x, E, red, lo, hi);
        st_relaxed_b128(tag_slot(d, red, c, lb), lo, hi);
      } else {
        ulonglong2* slot = reinterpret_cast<ulonglong2*>(part_slot(d, red, c, lb));
        slot[0] = make_ulonglong2((unsigned long long)x, (unsigned long long)(x >> 64));
        slot[1] = make_ulonglong2((unsigned long long)E, 0ull);
      }
    }
  }
}

// One warp: the total over the group's blocks of component c of reduction
// `red`, as a double on every lane.  All slot loads are issued before any is
// used; each lane folds its blocks in a fixed order, so every block of the
// group computes the same bits.
__device__ __forceinline__ double group_total(const Desc& d, int red, int c) {
  constexpr int PRE = 8;  // slots per lane held in registers (groups of up to 256 blocks per pass)
  const int lane = threadIdx.x & 31;
  fx::I128 acc = 0;
  int Ea = 1;
  for (int base = 0; base < d.nblk; base += 32 * PRE) {
    ulonglong2 w0[PRE];
    int ex[PRE];
#pragma unroll
    for (int t = 0; t < PRE; ++t) {
      const int j = base + lane + 32 * t;
      if (j < d.nblk) {
        const ulonglong2* slot = reinterpret_cast<const ulonglong2*>(part_slot(d, red, c, j));
        w0[t] = __ldcg(slot);
        ex[t] = (int)__ldcg(reinterpret_cast<const unsigned long long*>(slot + 1));
      } else {
        w0[t] = make_ulonglong2(0ull, 0ull);
        ex[t] = 1;
      }
    }
    int e = Ea;
#pragma unroll
    for (int t = 0; t < PRE; ++t) e = max(e, ex[t]);
    fx::I128 a = fx::sar(acc, e - Ea);
#pragma unroll
    for (int t = 0; t < PRE; ++t) {
      const fx::I128 x = ((fx::I128)(long long)w0[t].y << 64) | (fx::I128)w0[t].x;
      a += fx::sar(x, e - ex[t]);
    }
    acc = a;
    Ea = e;
  }
  const int E = (int)__reduce_max_sync(0xffffffffu, (unsigned)Ea);
  const fx::I128 t = warp_sum_i128(E < fx::kBadExp ? fx::sar(acc, E - Ea) : (fx::I128)0);
  return fx::to_double(t, E);
}

// Warps 0 .. NC-1 fetch one component each into sh.tot.
template <int NC>
__device__ __forceinline__ void totals_to_shared(const Desc& d, int red, Shared& sh) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < NC; c += nw) {
    const double t = group_total(d, red, c);
    if ((threadIdx.x & 31) == 0) sh.tot[c] = t;
  }
}

// After a barrier: totals of reduction `red`, identical in every block.
template <int NC>
__device__ __forceinline__ void get_totals(const Desc& d, int red, Shared& sh) {
  totals_to_shared<NC>(d, red, sh);
  __syncthreads();
}

// As get_totals, then `derive(sh)` runs on one thread to turn the totals
// into the scalars of the next phase (divisions are done once per block, not
// once per thread); all threads see them afterwards.  The warps that fetched
// the components meet on a named barrier before the derivation.
template <int NC, typename F>
__device__ __forceinline__ void get_totals_then(const Desc& d, int red, Shared& sh, F derive) {
  totals_to_shared<NC>(d, red, sh);
  const int nw = blockDim.x >> 5;
  const int wk = NC < nw ? NC : nw;
  if (wk > 1 && (int)(threadIdx.x >> 5) < wk) asm volatile("bar.sync 1, %0;" ::"r"(wk * 32) : "memory");
  if (threadIdx.x == 0) derive(sh);
  __syncthreads();
}

// One warp: wait until every block of the group has stored component c of
// reduction `red` in its tagged slot, then fold the slots as group_total does
// (fixed order, identical bits in every block).  Each lane polls its slots
// with relaxed loads, re-reading only those that did not yet carry the tag,
// so the polling load on the slots' cache lines falls as blocks arrive.
// (Visibility of the other blocks' published vectors comes from the group
// barrier, not from these loads.)  Gives up (false on every lane) after
// d.spin_ns of wall-clock time or when another block has given up.
__device__ __forceinline__ bool tagged_total(const Desc& d, int red, int c, double& total) {
  constexpr int PRE = 8;  // slots per lane per pass (groups of up to 256 blocks per pass)
  const int lane = threadIdx.x & 31;
  int* const timeout = &d.res->timeout;
  fx::I128 acc = 0;
  int Ea = 1;
  unsigned long long t0 = 0;
  unsigned spins = 0;
  for (int base = 0; base < d.nblk; base += 32 * PRE) {
    ulonglong2 w[PRE];
    unsigned pend = 0;   // slots of this lane still without the tag
#pragma unroll
    for (int t = 0; t < PRE; ++t) {
      w[t] = make_ulonglong2(0ull, 1ull << 24);  // m = 0, E = 1 for slots past the group
      if (base + lane + 32 * t < d.nblk) pend |= 1u << t;
    }
    while (true) {
      // every load of the round is issued before any is examined (a pending
      // slot's word is overwritten; a tagged one is kept)
      const unsigned pm = pend;
#pragma unroll
      for (int t = 0; t < PRE; ++t)
        if (pm & (1u << t)) w[t] = ld_relaxed_b128(tag_slot(d, red, c, base + lane + 32 * t));
#pragma unroll
      for (int t = 0; t < PRE; ++t)
        if ((pm & (1u << t)) && fx::tagged_current(w[t].x, w[t].y, red)) pend &= ~(1u << t);
      if (__all_sync(0xffffffffu, pend == 0)) break;
      if ((++spins & 63u) == 0) {
        int give_up = 0;
        if (lane == 0) {
          if (*(volatile int*)timeout) {
            give_up = 1;
          } else {
            const unsigned long long now = global_ns();
            if (t0 == 0) {
              t0 = now;
            } else if ((long long)(now - t0) > d.spin_ns) {
              atomicExch(timeout, 1);
              give_up = 1;
            }
          }
        }
        if (__shfl_sync(0xffffffffu, give_up, 0)) return false;
      }
    }
    int ex[PRE];
    int e = Ea;
#pragma unroll
    for (int t = 0; t < PRE; ++t) {
      ex[t] = fx::tagged_exponent(w[t].y);
      e = max(e, ex[t]);
    }
    fx::I128 a = fx::sar(acc, e - Ea);
#pragma unroll
    for (int t = 0; t < PRE; ++t) {
      a += fx::sar(fx::tagged_mantissa(w[t].x, w[t].y), e - ex[t]);
    }
    acc = a;
    Ea = e;
  }
  const int E = (int)__reduce_max_sync(0xffffffffu, (unsigned)Ea);
  const fx::I128 t = warp_sum_i128(E < fx::kBadExp ? fx::sar(acc, E - Ea) : (fx::I128)0);
  total = E < fx::kBadExp ? fx::to_double(t, E + fx::kTagShift) : fx::to_double(0, fx::kBadExp);
  return true;
}

// One reduction of the FP64 single-reduction solver.  red_start publishes
// the block's partials and arrives at the group barrier; work between the two
// calls overlaps the other blocks' arrival and must not write what other
// blocks read.  red_finish waits for the barrier (which makes the other
// blocks' published vectors visible), leaves the totals in sh.tot, runs
// stage() on every thread and derive(sh) on thread 0.
//
// Untagged, the slots are read after the barrier: two global round trips
// after the last block arrives.  Tagged (d.tagged), warps 0 .. NC-1 poll the
// slots while another thread waits on the barrier, so the totals are known
// when the barrier completes.
template <int NC>
__device__ __forceinline__ void red_start(const Desc& d, Group& grp, int lb, int red, double (&v)[NC], Shared& sh) {
  if (d.tagged) put_partials<NC, true>(d, lb, red, v, sh);
  else put_partials<NC>(d, lb, red, v, sh);
  grp.arrive();
}

template <int NC, typename F, typename G>
__device__ __forceinline__ bool red_finish(const Desc& d, Group& grp, int red, Shared& sh, F derive, G stage) {
  if (!d.tagged) {
    if (!grp.wait(sh)) return false;
    stage();
    get_totals_then<NC>(d, red, sh, derive);
    return true;
  }
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < NC; c += nw) {
    double t;
    if (!tagged_total(d, red, c, t)) {
      if ((threadIdx.x & 31) == 0) sh.tflag = 0;
      break;
    }
    if ((threadIdx.x & 31) == 0) sh.tot[c] = t;
  }
  // the barrier wait: lane 0 of the first warp that polls no slots (thread 0 after its slots otherwise)
  if (threadIdx.x == (nw > NC ? 32 * NC : 0) && !grp.wait_one()) sh.tflag = 0;
  __syncthreads();
  if (!sh.tflag) return false;
  stage();
  if (threadIdx.x == 0) derive(sh);
  __syncthreads();
  return true;
}

template <int NC>
__device__ __forceinline__ bool red_finish(const Desc& d, Group& grp, int red, Shared& sh) {
  return red_finish<NC>(d, grp, red, sh, [](Shared&) {}, [] {});
}

__device__ void finish(const Desc& d, int lb, int status, int its, int sweeps, double rel_rec, double rel_true,
                       double bnorm) {
  if (lb == 0 && threadIdx.x == 0) {
    d.res->t_end = global_ns();
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

// Own-row storage of one block: in shared memory (RES) or in global scratch.
struct Local {
  double* x;
  double* r;
  double* z;
  double* p;
  double* q;
  const double* di;
  double* bp;
  const int* row;     // [nloc + 1] offsets into col / val
  const int* col;
  const double* val;
};

// Row-wise SpMV over the block's own rows with T lanes per row.  Column j of
// an own row reads own(j - r0) when j is owned by this block and halo(j)
// (a value published by another block) otherwise.  op(il, s) receives
// s = (A v)_{r0 + il} on lane 0 of the row's group.
template <int T, typename V, typename FOwn, typename FHalo, typename Op>
__device__ __forceinline__ void spmv_local(const Local& L, int r0, int nloc, FOwn own, FHalo halo, Op op) {
  const int g = threadIdx.x / T, l = threadIdx.x % T, ng = blockDim.x / T;
  for (int base = 0; base < nloc; base += ng) {
    const int il = base + g;
    V s = V(0);
    if (il < nloc) {
      const int k1 = L.row[il + 1];
      for (int k = L.row[il] + l; k < k1; k += T) {
        const int jl = L.col[k] - r0;
        const V v = ((unsigned)jl < (unsigned)nloc) ? own(jl) : halo(jl + r0);
        s = fma(L.val[k], v, s);
      }
    }
    if (T > 1) {
#pragma unroll
      for (int o = T / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, T);
    }
    if (il < nloc && l == 0) op(il, s);
  }
}

// SpMV over the block's own rows when every column has been renumbered into
// the block's local space (own rows, then gathered halo values): all reads
// are shared-memory reads, no branch per entry.
template <int T, typename Op>
__device__ __forceinline__ void spmv_ext(const int* __restrict__ row, const int* __restrict__ col,
                                         const double* __restrict__ val, const double* ext, int nloc, Op op) {
  const int g = threadIdx.x / T, l = threadIdx.x % T, ng = blockDim.x / T;
  for (int base = 0; base < nloc; base += ng) {
    const int il = base + g;
    double s = 0.0;
    if (il < nloc) {
      const int k1 = row[il + 1];
      for (int k = row[il] + l; k < k1; k += T) s = fma(val[k], ext[col[k]], s);
    }
    if (T > 1) {
#pragma unroll
      for (int o = T / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, T);
    }
    if (il < nloc && l == 0) op(il, s);
  }
}

// FP64 Jacobi-PCG with two group barriers per iteration.
//
// p is kept twice: each block updates its own rows (p = z + beta p) and
// publishes them to the buffer of the iteration's parity; a block that needs
// p_j of a row it does not own recomputes z_j + beta p_j from the published
// z and the previous iteration's buffer, with the same fused multiply-add the
// owner used, so both see bit-identical values and the update needs no
// barrier of its own.
//
// RES: the block's CSR rows (columns renumbered by the halo plan), its
// vectors and a gather buffer for its halo live in shared memory for the
// whole solve.  Each product first gathers every halo value the block needs
// with independent loads, then runs from shared memory only.  Without RES
// the rows and vectors stay in global scratch and halo values are read in
// place.
template <int T, bool RES>
__device__ void solve_fp64(const Desc& d, int lb, Shared& sh) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int tid = threadIdx.x, bd = blockDim.x;
  const int chunk = (d.n + d.nblk - 1) / d.nblk;
  const int r0 = min(d.n, lb * chunk), r1 = min(d.n, r0 + chunk), nloc = r1 - r0;
  Group grp{d.bar, &d.res->timeout, (unsigned)d.nblk, 0u, d.spin_ns};
  int red = 0;

  Local L;
  double* pe = nullptr;     // RES: [own p | halo values]
  const int* hid = nullptr; // RES: global index of each halo slot
  int nh = 0;
  if constexpr (RES) {
    double* base = reinterpret_cast<double*>(dsm);
    L.x = base;
    L.r = base + chunk;
    L.z = base + 2 * chunk;
    L.q = base + 3 * chunk;
    double* di = base + 4 * chunk;
    L.bp = base + 5 * chunk;
    pe = base + 6 * chunk;
    L.p = pe;
    double* val = pe + chunk + d.halo_cap;
    int* row = reinterpret_cast<int*>(val + d.res_nnz_cap);
    int* col = row + chunk + 1;
    int* hidw = col + d.res_nnz_cap;
    const int k0 = nloc > 0 ? d.rowptr[r0] : 0;
    const int nnzl = nloc > 0 ? d.rowptr[r1] - k0 : 0;
    const int h0 = d.hptr[lb];
    nh = d.hptr[lb + 1] - h0;
    for (int i = tid; i <= nloc; i += bd) row[i] = d.rowptr[r0 + i] - k0;
    for (int k = tid; k < nnzl; k += bd) {
      col[k] = d.lcol[k0 + k];
      val[k] = d.val[k0 + k];
    }
    for (int h = tid; h < nh; h += bd) hidw[h] = d.hidx[h0 + h];
    for (int i = tid; i < nloc; i += bd) di[i] = d.dinv[r0 + i];
    L.di = di;
    L.row = row;
    L.col = col;
    L.val = val;
    hid = hidw;
  } else {
    L.x = d.x + r0;
    L.r = d.r + r0;
    L.z = d.z + r0;
    L.p = nullptr;
    L.q = d.q + r0;
    L.di = d.dinv + r0;
    L.bp = d.bp + r0;
    L.row = d.rowptr + r0;
    L.col = d.col;
    L.val = d.val;
  }

  // ---- means of b and x0 ----
  {
    double v2[2] = {0.0, 0.0};
    for (int i = tid; i < nloc; i += bd) {
      v2[0] += d.b[r0 + i];
      if (d.use_x0) v2[1] += d.x[r0 + i];
    }
    put_partials<2>(d, lb, red, v2, sh);
    if (!grp.sync(sh)) return;
    get_totals<2>(d, red, sh);
    ++red;
  }
  const double mb = d.fixed ? 0.0 : sh.tot[0] / d.n, mx = d.fixed ? 0.0 : sh.tot[1] / d.n;
  // ---- projected b and x0; x0 published for the first product ----
  {
    double v1[1] = {0.0};
    for (int i = tid; i < nloc; i += bd) {
      const double bi = is_fixed(d, r0 + i) ? 0.0 : d.b[r0 + i] - mb;
      L.bp[i] = bi;
      v1[0] += bi * bi;
      const double xi = (d.use_x0 && !is_fixed(d, r0 + i)) ? d.x[r0 + i] - mx : 0.0;
      L.x[i] = xi;
      if (RES) {
        d.x[r0 + i] = xi;
        pe[i] = xi;
      }
    }
    put_partials<1>(d, lb, red, v1, sh);
    if (!grp.sync(sh)) return;
    get_totals<1>(d, red, sh);
    ++red;
  }
  const double bnorm = sqrt(sh.tot[0]);
  if (!isfinite(bnorm)) { finish(d, lb, CGP_ERR_NONFINITE, 0, 0, 0.0, 0.0, bnorm); return; }
  if (bnorm == 0.0) {
    for (int i = tid; i < nloc; i += bd) d.x[r0 + i] = 0.0;
    finish(d, lb, CGP_OK, 0, 0, 0.0, 0.0, 0.0);
    return;
  }
  // ---- r = bp - K x0, z = D^-1 r, p = z (published to buffer 0) ----
  double v2init[2];
  {
    double v2[2] = {0.0, 0.0};
    auto op = [&](int il, double s) {
      const double ri = L.bp[il] - s;
      const double zi = L.di[il] * ri;
      L.r[il] = ri;
      L.z[il] = zi;
      if (RES) d.z[r0 + il] = zi;
      d.p[r0 + il] = zi;
      v2[0] += ri * zi;
      v2[1] += ri * ri;
    };
    if constexpr (RES) {
      for (int h = tid; h < nh; h += bd) pe[nloc + h] = __ldcg(d.x + hid[h]);
      __syncthreads();
      spmv_ext<T>(L.row, L.col, L.val, pe, nloc, op);
      __syncthreads();
      for (int i = tid; i < nloc; i += bd) pe[i] = L.z[i];
    } else {
      spmv_local<T, double>(
          L, r0, nloc, [&](int jl) { return L.x[jl]; }, [&](int j) { return __ldcg(d.x + j); }, op);
    }
    v2init[0] = v2[0];
    v2init[1] = v2[1];
  }
  int k = 0, status = CGP_ERR_NOT_CONVERGED;
  if (tid == 0) {
    const double stop = d.tol * bnorm;
    sh.sc[4] = stop * stop;    // the test ||r||^2 <= (tol ||b||)^2 needs no square root
    sh.sc[3] = 0.0;            // 1 / (r, z) of the previous iteration
  }
  // one thread: convergence test and beta from (r,z) and (r,r); everyone reads the outcome
  // kd: iterations completed when the reduction's values are current
  int kd = 0;
  auto derive_rz = [&](Shared& S) {
    const double rz = S.tot[0], rr = S.tot[1];
    int st = -1;
    if (!isfinite(rr) || !isfinite(rz)) st = CGP_ERR_NONFINITE;
    else if (rr <= S.sc[4]) st = CGP_OK;
    else if (kd >= d.max_it) st = CGP_ERR_NOT_CONVERGED;
    S.isc[0] = st;
    S.sc[0] = rr;
    S.sc[1] = kd > 0 ? rz * S.sc[3] : 0.0;  // beta = (r,z) / (r,z)_old
    S.sc[2] = rz;
  };
  // the (r,z), (r,r) reduction of the initial residual
  put_partials<2>(d, lb, red, v2init, sh);
  if (!grp.sync(sh)) return;
  get_totals_then<2>(d, red, sh, derive_rz);
  ++red;
  while (true) {
    if (sh.isc[0] >= 0) { status = sh.isc[0]; break; }
    // one thread of another warp prepares 1 / (r,z) for the next beta, off the critical path
    if (tid == 32 || (bd == 32 && tid == 0)) sh.sc[3] = 1.0 / sh.sc[2];
    const double beta = sh.sc[1];
    double* pcur = (k & 1) ? d.p2 : d.p;
    const double* pold = (k & 1) ? d.p : d.p2;
    if (k > 0) {  // own rows: p = z + beta p, published to this iteration's buffer
      for (int i = tid; i < nloc; i += bd) {
        if (RES) {
          const double pi = fma(beta, pe[i], L.z[i]);
          pe[i] = pi;
          pcur[r0 + i] = pi;
        } else {
          pcur[r0 + i] = fma(beta, pold[r0 + i], L.z[i]);
        }
      }
    }
    {  // q = K p; rows owned elsewhere rebuild p_j from the published z_j and p_j
      double v1[1] = {0.0};
      const double* pown = RES ? pe : pcur + r0;
      auto op = [&](int il, double s) {
        L.q[il] = s;
        v1[0] += pown[il] * s;
      };
      if constexpr (RES) {
        for (int h = tid; h < nh; h += bd) {
          const int j = hid[h];
          pe[nloc + h] = k == 0 ? __ldcg(pcur + j) : fma(beta, __ldcg(pold + j), __ldcg(d.z + j));
        }
        __syncthreads();
        spmv_ext<T>(L.row, L.col, L.val, pe, nloc, op);
      } else {
        __syncthreads();
        spmv_local<T, double>(
            L, r0, nloc, [&](int jl) { return pown[jl]; },
            [&](int j) { return k == 0 ? __ldcg(pcur + j) : fma(beta, __ldcg(pold + j), __ldcg(d.z + j)); },
            op);
      }
      put_partials<1>(d, lb, red, v1, sh);
      if (!grp.sync(sh)) return;
      get_totals_then<1>(d, red, sh, [&](Shared& S) {
        const double pq = S.tot[0];
        S.isc[1] = (pq > 0.0) ? -1 : (isfinite(pq) ? CGP_ERR_BREAKDOWN : CGP_ERR_NONFINITE);
        S.sc[5] = S.sc[2] / pq;  // alpha
      });
      ++red;
    }
    if (sh.isc[1] >= 0) { status = sh.isc[1]; break; }
    const double alpha = sh.sc[5];
    {  // x += alpha p, r -= alpha q, z = D^-1 r (z published)
      double v2[2] = {0.0, 0.0};
      const double* pown = RES ? pe : pcur + r0;
      for (int i = tid; i < nloc; i += bd) {
        L.x[i] = fma(alpha, pown[i], L.x[i]);
        const double ri = fma(-alpha, L.q[i], L.r[i]);
        const double zi = L.di[i] * ri;
        L.r[i] = ri;
        L.z[i] = zi;
        if (RES) d.z[r0 + i] = zi;
        v2[0] += ri * zi;
        v2[1] += ri * ri;
      }
      kd = k + 1;
      put_partials<2>(d, lb, red, v2, sh);
      if (!grp.sync(sh)) return;
      get_totals_then<2>(d, red, sh, derive_rz);
      ++red;
    }
    ++k;
  }
  // ---- x -= mean(x), published; true residual ----
  {
    double v1[1] = {0.0};
    for (int i = tid; i < nloc; i += bd) v1[0] += L.x[i];
    put_partials<1>(d, lb, red, v1, sh);
    if (!grp.sync(sh)) return;
    get_totals<1>(d, red, sh);
    ++red;
  }
  const double mxf = d.fixed ? 0.0 : sh.tot[0] / d.n;
  for (int i = tid; i < nloc; i += bd) {
    const double xi = L.x[i] - mxf;
    L.x[i] = xi;
    if (RES) {
      d.x[r0 + i] = xi;
      pe[i] = xi;
    }
  }
  if (!grp.sync(sh)) return;
  {
    double v1[1] = {0.0};
    auto op = [&](int il, double s) {
      const double t = L.bp[il] - s;
      v1[0] += t * t;
    };
    if constexpr (RES) {
      for (int h = tid; h < nh; h += bd) pe[nloc + h] = __ldcg(d.x + hid[h]);
      __syncthreads();
      spmv_ext<T>(L.row, L.col, L.val, pe, nloc, op);
    } else {
      spmv_local<T, double>(
          L, r0, nloc, [&](int jl) { return L.x[jl]; }, [&](int j) { return __ldcg(d.x + j); }, op);
    }
    put_partials<1>(d, lb, red, v1, sh);
    if (!grp.sync(sh)) return;
    get_totals<1>(d, red, sh);
    ++red;
  }
  finish(d, lb, status, k, 0, sqrt(sh.sc[0]) / bnorm, sqrt(sh.tot[0]) / bnorm, bnorm);
}

// FP64 Jacobi-PCG in the single-reduction form of Chronopoulos and Gear:
// one grid-wide reduction per iteration (red_start / red_finish; with tuning
// flag bit 3 its slots are tagged and read while the barrier fills).
//
// With u = D^-1 r and w = K u, the recurrences p = u + beta p and
// s = w + beta s (so that s = K p) replace the product K p, and (r,u),
// (w,u), (r,r) of an iteration share one reduction:
//   gamma = (r,u), delta = (w,u), beta = gamma / gamma_old,
//   alpha = gamma / (delta - beta gamma / alpha_old),
//   x += alpha p, r -= alpha s, u = D^-1 r, w = K u.
// The product w = K u needs u_j of rows owned by other blocks; each block
// rebuilds them from the owner's published r_j, w_j and s_j (two buffers of
// each, by iteration parity) with the owner's own operations, so both hold
// the same bits.
//
// The recurrences let the recursive residual drift from b - K x by
// rounding.  When the recursive residual meets the tolerance the solver
// projects x, forms the true residual, and restarts from it if that one
// does not meet the tolerance as well (at most kMaxRestarts times).
constexpr int kMaxRestarts = 16;

template <int T, bool RES>
__device__ void solve_fp64_sr(const Desc& d, int lb, Shared& sh) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int tid = threadIdx.x, bd = blockDim.x;
  const int chunk = (d.n + d.nblk - 1) / d.nblk;
  const int r0 = min(d.n, lb * chunk), r1 = min(d.n, r0 + chunk), nloc = r1 - r0;
  const size_t n = d.n;
  Group grp{d.bar, &d.res->timeout, (unsigned)d.nblk, 0u, d.spin_ns};
  int red = 0;

  // published buffers (global): R0/R1, W0/W1, S0/S1 by iteration parity
  double* const R0 = d.pub64;
  double* const R1 = d.pub64 + n;
  double* const W0 = d.pub64 + 2 * n;
  double* const W1 = d.pub64 + 3 * n;
  double* const S0 = d.pub64 + 4 * n;
  double* const S1 = d.pub64 + 5 * n;

  double *x, *r, *u, *w, *p, *s, *bp, *ext = nullptr;
  double* u2 = nullptr;   // RES: second buffer of u (u_k and u_(k+1) alternate)
  double *stR = nullptr, *stW = nullptr, *stS = nullptr;  // RES: staged halo r, w, s of the next iteration
  const double* di;
  const double* dih = nullptr;  // RES: D^-1 of the halo rows
  const int* hid = nullptr;     // RES: global index of each halo slot
  int nh = 0;
  Local L;  // row structure of the own rows
  if constexpr (RES) {
    double* base = reinterpret_cast<double*>(dsm);
    x = base;
    r = base + chunk;
    u = base + 2 * chunk;
    w = base + 3 * chunk;
    p = base + 4 * chunk;
    s = base + 5 * chunk;
    double* dil = base + 6 * chunk;
    bp = base + 7 * chunk;
    u2 = base + 8 * chunk;
    ext = base + 9 * chunk;                  // [chunk + halo_cap]: own u, then gathered halo u
    double* dh = ext + chunk + d.halo_cap;   // [halo_cap]
    double* val = dh + d.halo_cap;           // [nnz_cap]
    stR = val + d.res_nnz_cap;               // [halo_cap] each
    stW = stR + d.halo_cap;
    stS = stW + d.halo_cap;
    int* row = reinterpret_cast<int*>(stS + d.halo_cap);
    int* col = row + chunk + 1;
    int* hd = col + d.res_nnz_cap;
    const int k0 = nloc > 0 ? d.rowptr[r0] : 0;
    const int nnzl = nloc > 0 ? d.rowptr[r1] - k0 : 0;
    const int h0 = d.hptr[lb];
    nh = d.hptr[lb + 1] - h0;
    for (int i = tid; i <= nloc; i += bd) row[i] = d.rowptr[r0 + i] - k0;
    for (int k = tid; k < nnzl; k += bd) {
      col[k] = d.lcol[k0 + k];
      val[k] = d.val[k0 + k];
    }
    for (int h = tid; h < nh; h += bd) {
      const int j = d.hidx[h0 + h];
      hd[h] = j;
      dh[h] = d.dinv[j];
    }
    for (int i = tid; i < nloc; i += bd) dil[i] = d.dinv[r0 + i];
    di = dil;
    dih = dh;
    hid = hd;
    L.row = row;
    L.col = col;
    L.val = val;
  } else {
    x = d.x + r0;
    r = d.r + r0;
    u = d.z + r0;
    w = d.q + r0;
    p = d.p + r0;
    s = d.p2 + r0;
    bp = d.bp + r0;
    di = d.dinv + r0;
    L.row = d.rowptr + r0;
    L.col = d.col;
    L.val = d.val;
  }

  if (d.tagged) {
    if (!d.tpart) {   // the tagged slots are part of every mesh's scratch; a descriptor without them is a bug
      finish(d, lb, CGP_ERR_INVALID_ARG, 0, 0, 0.0, 0.0, 0.0);
      return;
    }
    // this block's tagged slots start empty; the group barrier of the first
    // reduction orders that before any block reads them
    if (tid < 6) *tag_slot(d, tid / 3, tid % 3, lb) = make_ulonglong2(0ull, 0ull);
  }
  // ---- means of b and x0 ----
  {
    double v2[2] = {0.0, 0.0};
    for (int i = tid; i < nloc; i += bd) {
      v2[0] += d.b[r0 + i];
      if (d.use_x0) v2[1] += d.x[r0 + i];
    }
    put_partials<2>(d, lb, red, v2, sh);
    if (!grp.sync(sh)) return;
    get_totals<2>(d, red, sh);
    ++red;
  }
  // ---- projected b and x0; x0 published for the first product ----
  {
    const double mb = d.fixed ? 0.0 : sh.tot[0] / d.n, mx = d.fixed ? 0.0 : sh.tot[1] / d.n;
    double v1[1] = {0.0};
    for (int i = tid; i < nloc; i += bd) {
      const double bi = is_fixed(d, r0 + i) ? 0.0 : d.b[r0 + i] - mb;
      bp[i] = bi;
      v1[0] += bi * bi;
      const double xi = (d.use_x0 && !is_fixed(d, r0 + i)) ? d.x[r0 + i] - mx : 0.0;
      x[i] = xi;
      if (RES) d.x[r0 + i] = xi;
    }
    red_start<1>(d, grp, lb, red, v1, sh);
    if (!red_finish<1>(d, grp, red, sh)) return;
    ++red;
  }
  const double bnorm = sqrt(sh.tot[0]);
  if (!isfinite(bnorm)) { finish(d, lb, CGP_ERR_NONFINITE, 0, 0, 0.0, 0.0, bnorm); return; }
  if (bnorm == 0.0) {
    for (int i = tid; i < nloc; i += bd) d.x[r0 + i] = 0.0;
    finish(d, lb, CGP_OK, 0, 0, 0.0, 0.0, 0.0);
    return;
  }
  const double stop = d.tol * bnorm, stop2 = stop * stop;
  if (tid == 0) sh.sc[4] = stop2;   // the test ||r||^2 <= (tol ||b||)^2 needs no square root

  int its = 0, restarts = 0, status = CGP_ERR_NOT_CONVERGED, pending = -1;
  double rr_rec = 0.0, rr_true = 0.0;
  bool first = true;
  while (true) {
    // ---- true residual of the projected, published x: r = bp - K x, u = D^-1 r; r published ----
    {
      double v1[1] = {0.0};
      auto op = [&](int il, double sum) {
        const double t = bp[il] - sum;
        r[il] = t;
        u[il] = di[il] * t;
        R0[r0 + il] = t;
        v1[0] += t * t;
      };
      if constexpr (RES) {
        for (int i = tid; i < nloc; i += bd) ext[i] = x[i];
        for (int h = tid; h < nh; h += bd) ext[nloc + h] = __ldcg(d.x + hid[h]);
        __syncthreads();
        spmv_ext<T>(L.row, L.col, L.val, ext, nloc, op);
      } else {
        spmv_local<T, double>(
            L, r0, nloc, [&](int jl) { return x[jl]; }, [&](int j) { return __ldcg(d.x + j); }, op);
      }
      red_start<1>(d, grp, lb, red, v1, sh);
      if (!red_finish<1>(d, grp, red, sh)) return;   // also publishes r for the first product
      ++red;
    }
    rr_true = sh.tot[0];
    if (first) rr_rec = rr_true;
    if (!isfinite(rr_true)) { status = CGP_ERR_NONFINITE; break; }
    if (rr_true <= stop2) { status = CGP_OK; break; }
    if (pending >= 0) { status = pending; break; }
    if (its >= d.max_it || restarts >= kMaxRestarts) { status = CGP_ERR_NOT_CONVERGED; break; }
    if (!first) ++restarts;
    first = false;

    // ---- w = K u (halo u_j = D^-1_j r_j from the published r) and the first reduction ----
    {
      double v3[3] = {0.0, 0.0, 0.0};
      auto op = [&](int il, double sum) {
        w[il] = sum;
        W0[r0 + il] = sum;
        const double ui = u[il], ri = r[il];
        v3[0] += ri * ui;
        v3[1] += sum * ui;
        v3[2] += ri * ri;
      };
      if constexpr (RES) {
        for (int i = tid; i < nloc; i += bd) ext[i] = u[i];
        for (int h = tid; h < nh; h += bd) ext[nloc + h] = dih[h] * __ldcg(R0 + hid[h]);
        __syncthreads();
        spmv_ext<T>(L.row, L.col, L.val, ext, nloc, op);
      } else {
        __syncthreads();
        spmv_local<T, double>(
            L, r0, nloc, [&](int jl) { return u[jl]; }, [&](int j) { return d.dinv[j] * __ldcg(R0 + j); }, op);
      }
      red_start<3>(d, grp, lb, red, v3, sh);
    }
    // RES: as soon as the reduction's slots show that every block has published,
    // the threads above warp 2 load the halo inputs r_j, w_j, s_j of the coming
    // iteration (they do not depend on the scalars).  A thread's first HREG
    // entries go to registers and are consumed by the same thread after the
    // own-row update, so the loads overlap the derivation and that update; any
    // further entries go through shared memory.
    constexpr int TW = 3 * 32;
    constexpr int HREG = 2;
    const bool staged = RES && bd > TW;
    double hR[HREG], hW[HREG], hS[HREG];
#pragma unroll
    for (int q = 0; q < HREG; ++q) hR[q] = hW[q] = hS[q] = 0.0;
    auto stage = [&](int kk) {
      if (!staged || tid < TW) return;
      const double* Rc = (kk & 1) ? R1 : R0;
      const double* Wc = (kk & 1) ? W1 : W0;
      const double* Sc = (kk & 1) ? S1 : S0;
      const int hs = bd - TW;
      int h = tid - TW;
#pragma unroll
      for (int q = 0; q < HREG; ++q, h += hs) {
        if (h < nh) {
          const int j = hid[h];
          hR[q] = __ldcg(Rc + j);
          hW[q] = __ldcg(Wc + j);
          if (kk > 0) hS[q] = __ldcg(Sc + j);
        }
      }
      for (; h < nh; h += hs) {
        const int j = hid[h];
        stR[h] = __ldcg(Rc + j);
        stW[h] = __ldcg(Wc + j);
        if (kk > 0) stS[h] = __ldcg(Sc + j);
      }
    };
    // scalars (thread 0): sc[0] alpha, sc[1] beta, sc[2] gamma, sc[5] (r,r), isc[0] stop flag;
    // sc[3] = 1 / gamma_old and sc[6] = 1 / alpha_old are prepared off the critical path
    int k = 0;
    auto derive = [&](Shared& S) {
      const double g = S.tot[0], dl = S.tot[1], rr = S.tot[2];
      int st = -1;
      if (!isfinite(g) || !isfinite(dl) || !isfinite(rr)) st = CGP_ERR_NONFINITE;
      else if (rr <= S.sc[4]) st = CGP_OK;
      else if (its + k >= d.max_it) st = CGP_ERR_NOT_CONVERGED;
      double beta = 0.0, alpha;
      if (k == 0) {
        alpha = g / dl;
      } else {
        beta = g * S.sc[3];
        alpha = g / (dl - beta * g * S.sc[6]);
      }
      if (st < 0 && !(g > 0.0 && alpha > 0.0 && isfinite(alpha))) st = CGP_ERR_BREAKDOWN;
      S.isc[0] = st;
      S.sc[0] = alpha;
      S.sc[1] = beta;
      S.sc[2] = g;
      S.sc[5] = rr;
    };
    if (!red_finish<3>(d, grp, red, sh, derive, [&] { stage(0); })) return;
    ++red;
    while (true) {
      const int st = sh.isc[0];
      if (st >= 0) {
        if (st != CGP_OK) pending = st;
        break;
      }
      if (tid == 32 || (bd == 32 && tid == 0)) {
        sh.sc[3] = 1.0 / sh.sc[2];
        sh.sc[6] = 1.0 / sh.sc[0];
      }
      const double alpha = sh.sc[0], beta = sh.sc[1];
      const double* Rc = (k & 1) ? R1 : R0;
      const double* Wc = (k & 1) ? W1 : W0;
      const double* Sc = (k & 1) ? S1 : S0;
      double* Rn = (k & 1) ? R0 : R1;
      double* Wn = (k & 1) ? W0 : W1;
      double* Sn = (k & 1) ? S0 : S1;
      // RES: u_k stays in uc while u_(k+1) goes to un, so that p and x (off the
      // critical path) are updated while the reduction completes
      double* uc = (RES && (k & 1)) ? u2 : u;
      double* un = (RES && !(k & 1)) ? u2 : u;
      // own rows: s, r, u (and without RES p, x); r and s published
      for (int i = tid; i < nloc; i += bd) {
        const double si = k == 0 ? w[i] : fma(beta, s[i], w[i]);
        if (!RES) {
          const double pi = k == 0 ? u[i] : fma(beta, p[i], u[i]);
          p[i] = pi;
          x[i] = fma(alpha, pi, x[i]);
        }
        s[i] = si;
        const double ri = fma(-alpha, si, r[i]);
        r[i] = ri;
        const double ui = di[i] * ri;
        un[i] = ui;
        Rn[r0 + i] = ri;
        Sn[r0 + i] = si;
        if (RES) ext[i] = ui;
      }
      // halo: u_j = D^-1_j (r_j - alpha (w_j + beta s_j)) from the owner's published values
      auto halo_u = [&](int j, double dj) {
        const double sj = k == 0 ? __ldcg(Wc + j) : fma(beta, __ldcg(Sc + j), __ldcg(Wc + j));
        return dj * fma(-alpha, sj, __ldcg(Rc + j));
      };
      if constexpr (RES) {
        if (staged) {
          if (tid >= TW) {   // the entries this thread staged
            const int hs = bd - TW;
            int h = tid - TW;
#pragma unroll
            for (int q = 0; q < HREG; ++q, h += hs) {
              if (h < nh) {
                const double sj = k == 0 ? hW[q] : fma(beta, hS[q], hW[q]);
                ext[nloc + h] = dih[h] * fma(-alpha, sj, hR[q]);
              }
            }
            for (; h < nh; h += hs) {
              const double sj = k == 0 ? stW[h] : fma(beta, stS[h], stW[h]);
              ext[nloc + h] = dih[h] * fma(-alpha, sj, stR[h]);
            }
          }
        } else {
          for (int h = tid; h < nh; h += bd) ext[nloc + h] = halo_u(hid[h], dih[h]);
        }
      }
      __syncthreads();
      double v3[3] = {0.0, 0.0, 0.0};
      auto op = [&](int il, double sum) {
        w[il] = sum;
        Wn[r0 + il] = sum;
        const double ui = un[il], ri = r[il];
        v3[0] += ri * ui;
        v3[1] += sum * ui;
        v3[2] += ri * ri;
      };
      if constexpr (RES) {
        spmv_ext<T>(L.row, L.col, L.val, ext, nloc, op);
      } else {
        spmv_local<T, double>(
            L, r0, nloc, [&](int jl) { return un[jl]; }, [&](int j) { return halo_u(j, d.dinv[j]); }, op);
      }
      red_start<3>(d, grp, lb, red, v3, sh);
      if constexpr (RES) {   // p_k = u_k + beta p_(k-1), x += alpha p_k while the other blocks catch up
        for (int i = tid; i < nloc; i += bd) {
          const double pi = k == 0 ? uc[i] : fma(beta, p[i], uc[i]);
          p[i] = pi;
          x[i] = fma(alpha, pi, x[i]);
        }
      }
      ++k;
      if (!red_finish<3>(d, grp, red, sh, derive, [&] { stage(k); })) return;
      ++red;
    }
    its += k;
    rr_rec = sh.sc[5];
    // ---- x -= mean(x), published for the true residual ----
    {
      double v1[1] = {0.0};
      for (int i = tid; i < nloc; i += bd) v1[0] += x[i];
      red_start<1>(d, grp, lb, red, v1, sh);
      if (!red_finish<1>(d, grp, red, sh)) return;
      ++red;
    }
    const double mxf = d.fixed ? 0.0 : sh.tot[0] / d.n;
    for (int i = tid; i < nloc; i += bd) {
      const double xi = x[i] - mxf;
      x[i] = xi;
      if (RES) d.x[r0 + i] = xi;
    }
    if (!grp.sync(sh)) return;
  }
  finish(d, lb, status, its, restarts, sqrt(rr_rec) / bnorm, sqrt(rr_true) / bnorm, bnorm);
}

// ---------------------------------------------------------------------------
// FP32 reductions of the inner solve: warp trees on the FP32 pipe, one slot
// per block, every block sums the slots in the same order (deterministic).
// ---------------------------------------------------------------------------
template <int NC>
__device__ __forceinline__ void put_partials_f(const Desc& d, int lb, int red, const float (&v)[NC], Shared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const float s = warp_sum(v[c]);
    if (lane == 0) sh.fred[c][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float s = lane < nw ? sh.fred[c][lane] : 0.0f;
      s = warp_sum(s);
      if (lane == 0) d.fpart[((red & 1) * NCOMP + c) * d.part_stride + lb] = s;
    }
  }
}

template <int NC, typename F>
__device__ __forceinline__ void get_totals_f_then(const Desc& d, int red, Shared& sh, F derive) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float* src = d.fpart + ((red & 1) * NCOMP + c) * d.part_stride;
      float s = 0.0f;
      for (int j = lane; j < d.nblk; j += 32) s += __ldcg(src + j);
      s = warp_sum(s);
      if (lane == 0) sh.ftot[c] = s;
    }
    if (lane == 0) derive(sh);
  }
  __syncthreads();
}

// FP32 SpMV over the block's rows reading the global CSR: own columns from
// own(jl), other columns from halo(j).
template <int T, typename FOwn, typename FHalo, typename Op>
__device__ __forceinline__ void spmv_local_f(const int* __restrict__ row, const int* __restrict__ col,
                                             const float* __restrict__ val, int r0, int nloc, FOwn own,
                                             FHalo halo, Op op) {
  const int g = threadIdx.x / T, l = threadIdx.x % T, ng = blockDim.x / T;
  for (int base = 0; base < nloc; base += ng) {
    const int il = base + g;
    float s = 0.0f;
    if (il < nloc) {
      const int k1 = row[il + 1];
      for (int k = row[il] + l; k < k1; k += T) {
        const int jl = col[k] - r0;
        const float v = ((unsigned)jl < (unsigned)nloc) ? own(jl) : halo(jl + r0);
        s = fmaf(val[k], v, s);
      }
    }
    if (T > 1) {
#pragma unroll
      for (int o = T / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, T);
    }
    if (il < nloc && l == 0) op(il, s);
  }
}

// FP32 SpMV over the block's rows with a gathered local vector (RES) or with
// halo values computed on the fly from published buffers (no RES).
template <int T, typename Op>
__device__ __forceinline__ void spmv_ext32(const int* __restrict__ row, const int* __restrict__ col,
                                           const float* __restrict__ val, const float* ext, int nloc, Op op) {
  const int g = threadIdx.x / T, l = threadIdx.x % T, ng = blockDim.x / T;
  for (int base = 0; base < nloc; base += ng) {
    const int il = base + g;
    float s = 0.0f;
    if (il < nloc) {
      const int k1 = row[il + 1];
      for (int k = row[il] + l; k < k1; k += T) s = fmaf(val[k], ext[col[k]], s);
    }
    if (T > 1) {
#pragma unroll
      for (int o = T / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, T);
    }
    if (il < nloc && l == 0) op(il, s);
  }
}

// Mixed precision: FP64 iterative refinement around FP32 inner solves.
//
// Outer (FP64, global memory): r = bp - K x, r -= mean(r), stop when
// ||r|| <= tol ||bp||; after each inner solve x += e, x -= mean(x).
// Inner (FP32): Jacobi-preconditioned CG in the single-reduction form of
// Chronopoulos and Gear (the recurrence s = w + beta s replaces the product
// A p, and (r,u), (w,u), (r,r) share one reduction), solving K e = r from
// e = 0 to ||r_inner|| <= max(inner_tol ||r||, tol ||b|| / 2).  One barrier per inner
// iteration: the product w = A u needs u_j of rows owned elsewhere, which
// each block rebuilds from the owner's published r_j, w_j, s_j (kept in two
// buffers by iteration parity) with the owner's own FMAs.
template <int T, bool RES>
__device__ void solve_mixed(const Desc& d, int lb, Shared& sh) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int tid = threadIdx.x, bd = blockDim.x;
  const int chunk = (d.n + d.nblk - 1) / d.nblk;
  const int r0 = min(d.n, lb * chunk), r1 = min(d.n, r0 + chunk), nloc = r1 - r0;
  const size_t n = d.n;
  Group grp{d.bar, &d.res->timeout, (unsigned)d.nblk, 0u, d.spin_ns};
  int red = 0;

  // published buffers (global): R0/R1, W0/W1, S0/S1 by iteration parity
  float* const R0 = d.f32pub;
  float* const R1 = d.f32pub + n;
  float* const W0 = d.f32pub + 2 * n;
  float* const W1 = d.f32pub + 3 * n;
  float* const S0 = d.f32pub + 4 * n;
  float* const S1 = d.f32pub + 5 * n;
  // own inner vectors and the local system
  float *ir, *iu, *iw, *ip, *is, *ie, *ext = nullptr, *dih = nullptr;
  float *stR = nullptr, *stW = nullptr, *stS = nullptr;   // RES: staged halo r, w, s of the next iteration
  const float* di;
  const int *row, *col, *hid = nullptr;
  const float* val;
  int nh = 0;
  if constexpr (RES) {
    float* f = reinterpret_cast<float*>(dsm);
    ir = f;
    iu = f + chunk;
    iw = f + 2 * chunk;
    ip = f + 3 * chunk;
    is = f + 4 * chunk;
    ie = f + 5 * chunk;
    float* dil = f + 6 * chunk;
    ext = f + 7 * chunk;                   // [chunk + halo_cap]
    dih = ext + chunk + d.halo_cap;        // [halo_cap]
    float* vl = dih + d.halo_cap;          // [nnz_cap]
    stR = vl + d.res_nnz_cap;              // [halo_cap] each
    stW = stR + d.halo_cap;
    stS = stW + d.halo_cap;
    int* rw = reinterpret_cast<int*>(stS + d.halo_cap);
    int* cl = rw + chunk + 1;
    int* hd = cl + d.res_nnz_cap;
    const int k0 = nloc > 0 ? d.rowptr[r0] : 0;
    const int nnzl = nloc > 0 ? d.rowptr[r1] - k0 : 0;
    const int h0 = d.hptr[lb];
    nh = d.hptr[lb + 1] - h0;
    for (int i = tid; i <= nloc; i += bd) rw[i] = d.rowptr[r0 + i] - k0;
    for (int k = tid; k < nnzl; k += bd) {
      cl[k] = d.lcol[k0 + k];
      vl[k] = d.val32[k0 + k];
    }
    for (int h = tid; h < nh; h += bd) {
      const int j = d.hidx[h0 + h];
      hd[h] = j;
      dih[h] = d.dinv32[j];
    }
    for (int i = tid; i < nloc; i += bd) dil[i] = d.dinv32[r0 + i];
    di = dil;
    row = rw;
    col = cl;
    val = vl;
    hid = hd;
  } else {
    float* o = d.f32own;
    ir = o + r0;
    iu = o + n + r0;
    iw = o + 2 * n + r0;
    ip = o + 3 * n + r0;
    is = o + 4 * n + r0;
    ie = o + 5 * n + r0;
    di = d.dinv32 + r0;
    row = d.rowptr + r0;
    col = d.col;
    val = d.val32;
  }
  // outer FP64 storage (global)
  double* x = d.x + r0;
  double* bp = d.bp + r0;
  double* r64 = d.r + r0;

  // ---- projected b and x0 ----
  {
    double v2[2] = {0.0, 0.0};
    for (int i = tid; i < nloc; i += bd) {
      v2[0] += d.b[r0 + i];
      if (d.use_x0) v2[1] += x[i];
    }
    put_partials<2>(d, lb, red, v2, sh);
    if (!grp.sync(sh)) return;
    get_totals<2>(d, red, sh);
    ++red;
  }
  {
    const double mb = d.fixed ? 0.0 : sh.tot[0] / d.n, mx = d.fixed ? 0.0 : sh.tot[1] / d.n;
    double v1[1] = {0.0};
    for (int i = tid; i < nloc; i += bd) {
      const double bi = is_fixed(d, r0 + i) ? 0.0 : d.b[r0 + i] - mb;
      bp[i] = bi;
      v1[0] += bi * bi;
      x[i] = (d.use_x0 && !is_fixed(d, r0 + i)) ? x[i] - mx : 0.0;
    }
    put_partials<1>(d, lb, red, v1, sh);
    if (!grp.sync(sh)) return;
    get_totals<1>(d, red, sh);
    ++red;
  }
  const double bnorm = sqrt(sh.tot[0]);
  if (!isfinite(bnorm)) { finish(d, lb, CGP_ERR_NONFINITE, 0, 0, 0.0, 0.0, bnorm); return; }
  if (bnorm == 0.0) {
    for (int i = tid; i < nloc; i += bd) x[i] = 0.0;
    finish(d, lb, CGP_OK, 0, 0, 0.0, 0.0, 0.0);
    return;
  }
  // FP64 view of the local rows for the outer residual (global arrays)
  Local L;
  L.row = d.rowptr + r0;
  L.col = d.col;
  L.val = d.val;

  int total = 0, sweeps = 0, status = CGP_ERR_NOT_CONVERGED;
  double rel = 0.0;
  while (true) {
    // ---- FP64 residual r = bp - K x, projected; x is complete (barrier above) ----
    {
      double v1[1] = {0.0};
      spmv_local<T, double>(
          L, r0, nloc, [&](int jl) { return x[jl]; }, [&](int j) { return __ldcg(d.x + j); },
          [&](int il, double s) {
            const double ri = bp[il] - s;
            r64[il] = ri;
            v1[0] += ri;
          });
      put_partials<1>(d, lb, red, v1, sh);
      if (!grp.sync(sh)) return;
      get_totals<1>(d, red, sh);
      ++red;
    }
    {
      const double mr = d.fixed ? 0.0 : sh.tot[0] / d.n;
      double v1[1] = {0.0};
      for (int i = tid; i < nloc; i += bd) {
        const double ri = r64[i] - mr;
        v1[0] += ri * ri;
        const float rf = (float)ri;
        ir[i] = rf;
        iu[i] = di[i] * rf;
        ie[i] = 0.0f;
        R0[r0 + i] = rf;
      }
      put_partials<1>(d, lb, red, v1, sh);
      if (!grp.sync(sh)) return;   // also publishes r_0 for the first product
      get_totals<1>(d, red, sh);
      ++red;
    }
    rel = sqrt(sh.tot[0]) / bnorm;
    if (!isfinite(rel)) { status = CGP_ERR_NONFINITE; break; }
    if (rel <= d.tol) { status = CGP_OK; break; }
    if (sweeps >= d.max_sweeps || total >= d.max_it) { status = CGP_ERR_NOT_CONVERGED; break; }

    // ---- FP32 inner solve, single-reduction CG ----
    // w_0 = A u_0 (u_j = D^-1_j r_j from the published r_0)
    if constexpr (RES) {
      for (int i = tid; i < nloc; i += bd) ext[i] = iu[i];
      for (int h = tid; h < nh; h += bd) ext[nloc + h] = dih[h] * __ldcg(R0 + hid[h]);
      __syncthreads();
    }
    {
      float v3[3] = {0.0f, 0.0f, 0.0f};
      auto op = [&](int il, float s) {
        iw[il] = s;
        W0[r0 + il] = s;
        const float u = iu[il], r = ir[il];
        v3[0] = fmaf(r, u, v3[0]);
        v3[1] = fmaf(s, u, v3[1]);
        v3[2] = fmaf(r, r, v3[2]);
      };
      if constexpr (RES) {
        spmv_ext32<T>(row, col, val, ext, nloc, op);
      } else {
        spmv_local_f<T>(row, col, val, r0, nloc, [&](int jl) { return iu[jl]; },
                        [&](int j) { return d.dinv32[j] * __ldcg(R0 + j); }, op);
      }
      put_partials_f<3>(d, lb, red, v3, sh);
      if (!grp.sync(sh)) return;
    }
    // scalars (thread 0): sc[0] alpha, sc[1] beta, sc[2] gamma, isc[0] stop flag
    int k = 0;
    auto derive = [&](Shared& S) {
      const float g = S.ftot[0], dl = S.ftot[1], rr = S.ftot[2];
      int st = -1;
      if (k == 0) S.fsc[3] = rr;                                       // ||r_0||^2 of this sweep
      if (!isfinite(rr) || !isfinite(g) || !isfinite(dl)) st = 1;     // non-finite
      else if (rr <= fmaxf(S.fsc[4] * S.fsc[3], S.fsc[5])) st = 0;   // inner tolerance reached
      else if (total + k >= d.max_it) st = 0;
      float beta = 0.0f, alpha;
      if (k == 0) {
        alpha = g / dl;
      } else {
        beta = g / S.fsc[2];
        alpha = g / (dl - beta * g / S.fsc[0]);
      }
      if (st < 0 && !(g > 0.0f && alpha > 0.0f && isfinite(alpha))) st = 2;  // breakdown
      S.isc[0] = st;
      S.fsc[0] = alpha;
      S.fsc[1] = beta;
      S.fsc[2] = g;
    };
    if (tid == 0) {
      sh.fsc[4] = (float)(d.inner_tol * d.inner_tol);
      // below half the outer target the correction would already pass the outer test
      const double floor = 0.5 * d.tol * bnorm;
      sh.fsc[5] = (float)(floor * floor);
    }
    // RES: while warp 0 fetches the reduction's totals, the other warps stage
    // the halo inputs r_j, w_j, s_j of the coming iteration, so the two global
    // round trips overlap
    const bool staged = RES && bd > 32;
    auto stage = [&](int kk) {
      if (!staged || tid < 32) return;
      const float* Rc = (kk & 1) ? R1 : R0;
      const float* Wc = (kk & 1) ? W1 : W0;
      const float* Sc = (kk & 1) ? S1 : S0;
      for (int h = tid - 32; h < nh; h += bd - 32) {
        const int j = hid[h];
        stR[h] = __ldcg(Rc + j);
        stW[h] = __ldcg(Wc + j);
        if (kk > 0) stS[h] = __ldcg(Sc + j);
      }
    };
    stage(0);
    get_totals_f_then<3>(d, red, sh, derive);
    ++red;
    bool bad = false;
    while (true) {
      const int st = sh.isc[0];
      if (st >= 0) {
        bad = st == 1;
        break;
      }
      const float alpha = sh.fsc[0], beta = sh.fsc[1];
      const float* Rc = (k & 1) ? R1 : R0;
      const float* Wc = (k & 1) ? W1 : W0;
      const float* Sc = (k & 1) ? S1 : S0;
      float* Rn = (k & 1) ? R0 : R1;
      float* Wn = (k & 1) ? W0 : W1;
      float* Sn = (k & 1) ? S0 : S1;
      // own rows: p, s, e, r, u
      for (int i = tid; i < nloc; i += bd) {
        const float pi = k == 0 ? iu[i] : fmaf(beta, ip[i], iu[i]);
        const float si = k == 0 ? iw[i] : fmaf(beta, is[i], iw[i]);
        ip[i] = pi;
        is[i] = si;
        ie[i] = fmaf(alpha, pi, ie[i]);
        const float ri = fmaf(-alpha, si, ir[i]);
        ir[i] = ri;
        iu[i] = di[i] * ri;
        Rn[r0 + i] = ri;
        Sn[r0 + i] = si;
        if (RES) ext[i] = di[i] * ri;
      }
      // halo: u_j = D^-1_j (r_j - alpha (w_j + beta s_j)) from the owner's published values
      auto halo_u = [&](int j, float dj) {
        const float sj = k == 0 ? __ldcg(Wc + j) : fmaf(beta, __ldcg(Sc + j), __ldcg(Wc + j));
        return dj * fmaf(-alpha, sj, __ldcg(Rc + j));
      };
      if constexpr (RES) {
        if (staged) {
          for (int h = tid; h < nh; h += bd) {
            const float sj = k == 0 ? stW[h] : fmaf(beta, stS[h], stW[h]);
            ext[nloc + h] = dih[h] * fmaf(-alpha, sj, stR[h]);
          }
        } else {
          for (int h = tid; h < nh; h += bd) ext[nloc + h] = halo_u(hid[h], dih[h]);
        }
      }
      __syncthreads();
      float v3[3] = {0.0f, 0.0f, 0.0f};
      auto op = [&](int il, float s) {
        iw[il] = s;
        Wn[r0 + il] = s;
        const float u = iu[il], r = ir[il];
        v3[0] = fmaf(r, u, v3[0]);
        v3[1] = fmaf(s, u, v3[1]);
        v3[2] = fmaf(r, r, v3[2]);
      };
      if constexpr (RES) {
        spmv_ext32<T>(row, col, val, ext, nloc, op);
      } else {
        spmv_local_f<T>(row, col, val, r0, nloc, [&](int jl) { return iu[jl]; },
                        [&](int j) { return halo_u(j, d.dinv32[j]); }, op);
      }
      put_partials_f<3>(d, lb, red, v3, sh);
      if (!grp.sync(sh)) return;
      ++k;
      stage(k);
      get_totals_f_then<3>(d, red, sh, derive);
      ++red;
    }
    total += k;
    if (bad) { status = CGP_ERR_NONFINITE; break; }
    // ---- FP64 correction and projection; x published for the next residual ----
    {
      double v1[1] = {0.0};
      for (int i = tid; i < nloc; i += bd) {
        const double xi = x[i] + (double)ie[i];
        x[i] = xi;
        v1[0] += xi;
      }
      put_partials<1>(d, lb, red, v1, sh);
      if (!grp.sync(sh)) return;
      get_totals<1>(d, red, sh);
      ++red;
      const double mx = d.fixed ? 0.0 : sh.tot[0] / d.n;
      for (int i = tid; i < nloc; i += bd) x[i] -= mx;
      if (!grp.sync(sh)) return;
    }
    ++sweeps;
    if (k == 0 && total < d.max_it) { status = CGP_ERR_BREAKDOWN; break; }  // no inner progress
  }
  finish(d, lb, status, total, sweeps, rel, rel, bnorm);
}

template <int T, bool RES>
__global__ void __launch_bounds__(MAX_BLOCK) pcg_persistent_kernel(Desc d) {
  __shared__ Shared sh;
  mark_pending(d, blockIdx.x);
  if (d.mixed)
    solve_mixed<T, RES>(d, blockIdx.x, sh);
  else if (d.classic)
    solve_fp64<T, RES>(d, blockIdx.x, sh);
  else
    solve_fp64_sr<T, RES>(d, blockIdx.x, sh);
}

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

PcgFn pcg_kernel_for(int lanes, bool res) {
  switch (lanes) {
    case 1: return res ? pcg_persistent_kernel<1, true> : pcg_persistent_kernel<1, false>;
    case 2: return res ? pcg_persistent_kernel<2, true> : pcg_persistent_kernel<2, false>;
    case 4: return res ? pcg_persistent_kernel<4, true> : pcg_persistent_kernel<4, false>;
    case 8: return res ? pcg_persistent_kernel<8, true> : pcg_persistent_kernel<8, false>;
    case 32: return res ? pcg_persistent_kernel<32, true> : pcg_persistent_kernel<32, false>;
    default: return nullptr;
  }
}

using BatchFn = void (*)(const Desc*, const int*, unsigned long long*);

BatchFn batched_kernel_for(int lanes, bool res) {
  switch (lanes) {
    case 1: return res ? pcg_batched_kernel<1, true> : pcg_batched_kernel<1, false>;
    case 2: return res ? pcg_batched_kernel<2, true> : pcg_batched_kernel<2, false>;
    case 4: return res ? pcg_batched_kernel<4, true> : pcg_batched_kernel<4, false>;
    case 8: return res ? pcg_batched_kernel<8, true> : pcg_batched_kernel<8, false>;
    case 32: return res ? pcg_batched_kernel<32, true> : pcg_batched_kernel<32, false>;
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

int coresident_blocks(PcgFn fn, int block, int device, size_t smem = 0) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, block, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * dev_info(device).sms;
}

int optin_smem(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  return v;
}

struct LaunchPlan {
  PcgFn fn = nullptr;
  int nblk = 1;
  int block = 512;
  size_t smem = 0;
  int nnz_cap = 0;
  int halo_cap = 0;
  bool res = false;
  HaloPlan halo;
};

// Build (once per block count) the row partition and halo lists of a mesh.
// Halo lists of a pattern split into nblk contiguous row chunks.
int build_halo_plan(const std::vector<int>& rp, const std::vector<int>& cl, int n, int nblk, HaloPlan& out) {
  const int nnz = rp[n];
  const int chunk = (n + nblk - 1) / nblk;
  std::vector<int> lcol(nnz), hptr(nblk + 1, 0), hidx, h;
  HaloPlan p;
  p.nblk = nblk;
  for (int b = 0; b < nblk; ++b) {
    const int r0 = std::min(n, b * chunk), r1 = std::min(n, r0 + chunk), nloc = r1 - r0;
    const int k0 = rp[r0], k1 = rp[r1];
    h.clear();
    for (int k = k0; k < k1; ++k)
      if (cl[k] < r0 || cl[k] >= r1) h.push_back(cl[k]);
    std::sort(h.begin(), h.end());
    h.erase(std::unique(h.begin(), h.end()), h.end());
    for (int k = k0; k < k1; ++k) {
      const int j = cl[k];
      lcol[k] = (j >= r0 && j < r1) ? j - r0
                                    : nloc + (int)(std::lower_bound(h.begin(), h.end(), j) - h.begin());
    }
    hptr[b + 1] = hptr[b] + (int)h.size();
    hidx.insert(hidx.end(), h.begin(), h.end());
    p.max_rows = std::max(p.max_rows, nloc);
    p.max_nnz = std::max(p.max_nnz, k1 - k0);
    p.max_halo = std::max(p.max_halo, (int)h.size());
  }
  const size_t b_lcol = (size_t)nnz * 4, b_hptr = (size_t)(nblk + 1) * 4, b_hidx = std::max<size_t>(1, hidx.size()) * 4;
  const size_t o_hptr = (b_lcol + 255) / 256 * 256, o_hidx = o_hptr + (b_hptr + 255) / 256 * 256;
  CGP_CUDA(cudaMalloc(&p.base, o_hidx + b_hidx));
  char* base = static_cast<char*>(p.base);
  p.lcol = (int*)base;
  p.hptr = (int*)(base + o_hptr);
  p.hidx = (int*)(base + o_hidx);
  cudaError_t e = cudaMemcpy(p.lcol, lcol.data(), b_lcol, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p.hptr, hptr.data(), b_hptr, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !hidx.empty()) e = cudaMemcpy(p.hidx, hidx.data(), hidx.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p.base);
    return cuda_fail(e, "cudaMemcpy(halo plan)");
  }
  out = p;
  return CGP_OK;
}

int get_halo_plan(cgp_mesh_impl* m, int nblk, HaloPlan& out) {
  for (const HaloPlan& p : m->plans)
    if (p.nblk == nblk) {
      out = p;
      return CGP_OK;
    }
  HaloPlan p;
  int st = build_halo_plan(m->h_rowptr, m->h_col, m->n_c, nblk, p);
  if (st != CGP_OK) return st;
  m->plans.push_back(p);
  out = p;
  return CGP_OK;
}

// Recursive coordinate bisection of the nodes idx[lo, hi) into k parts whose
// sizes follow the solver's chunking (every part `chunk` rows but the last):
// the left side takes k/2 parts, split along the wider side of the bounding
// box; ties broken by node index, so the partition is deterministic.
void rcb(std::vector<int>& idx, int lo, int hi, int k, int chunk, const std::vector<double>& xy) {
  if (k <= 1 || hi - lo <= 1) return;
  double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
  for (int q = lo; q < hi; ++q) {
    const double x = xy[2 * (size_t)idx[q]], y = xy[2 * (size_t)idx[q] + 1];
    x0 = std::min(x0, x); x1 = std::max(x1, x); y0 = std::min(y0, y); y1 = std::max(y1, y);
  }
  const int axis = (x1 - x0) >= (y1 - y0) ? 0 : 1;
  const int k1 = k / 2;
  const int mid = std::min(hi, lo + k1 * chunk);
  std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int a, int b) {
    const double va = xy[2 * (size_t)a + axis], vb = xy[2 * (size_t)b + axis];
    return va < vb || (va == vb && a < b);
  });
  rcb(idx, lo, mid, k1, chunk, xy);
  rcb(idx, mid, hi, k - k1, chunk, xy);
}

// The system of a solve on nblk blocks in the bisection order (built once per
// block count and boundary condition): permuted pattern, values, D^-1, the
// Dirichlet mask, b and x buffers in the new order, and its halo plan.
int get_perm_system(cgp_mesh_impl* m, int nblk, PermSystem*& out) {
  const int dir = m->far_dirichlet;
  for (PermSystem& ps : m->psys)
    if (ps.nblk == nblk && ps.dirichlet == dir) {
      out = &ps;
      return CGP_OK;
    }
  const int n = m->n_c, nnz = m->nnz, chunk = (n + nblk - 1) / nblk;
  std::vector<double> xy(2 * (size_t)n), K(nnz), dv(n);
  CGP_CUDA(cudaDeviceSynchronize());
  CGP_CUDA(cudaMemcpy(xy.data(), m->xy_c, xy.size() * 8, cudaMemcpyDeviceToHost));
  CGP_CUDA(cudaMemcpy(K.data(), dir ? m->Kd : m->K, (size_t)nnz * 8, cudaMemcpyDeviceToHost));
  CGP_CUDA(cudaMemcpy(dv.data(), dir ? m->dinvd : m->dinv, (size_t)n * 8, cudaMemcpyDeviceToHost));
  std::vector<unsigned char> fix;
  if (dir) {
    fix.resize(n);
    CGP_CUDA(cudaMemcpy(fix.data(), m->fixed, n, cudaMemcpyDeviceToHost));
  }
  std::vector<int> perm(n), inv(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  rcb(perm, 0, n, nblk, chunk, xy);
  for (int b = 0; b < nblk; ++b) {   // mesh order inside every chunk (locality of the slices)
    const int r0 = std::min(n, b * chunk), r1 = std::min(n, r0 + chunk);
    std::sort(perm.begin() + r0, perm.begin() + r1);
  }
  for (int i = 0; i < n; ++i) inv[perm[i]] = i;
  PermSystem ps;
  ps.nblk = nblk;
  ps.dirichlet = dir;
  ps.n = n;
  ps.h_rowptr.assign(n + 1, 0);
  ps.h_col.resize(nnz);
  std::vector<double> pk(nnz), pd(n);
  std::vector<float> pk32(nnz), pd32(n);
  std::vector<unsigned char> pfix(dir ? n : 0);
  std::vector<std::pair<int, double>> row;
  for (int r = 0; r < n; ++r) {
    const int o = perm[r];
    row.clear();
    for (int k = m->h_rowptr[o]; k < m->h_rowptr[o + 1]; ++k) row.push_back({inv[m->h_col[k]], K[k]});
    std::sort(row.begin(), row.end());
    const int k0 = ps.h_rowptr[r];
    for (size_t q = 0; q < row.size(); ++q) {
      ps.h_col[k0 + q] = row[q].first;
      pk[k0 + q] = row[q].second;
      pk32[k0 + q] = (float)row[q].second;
    }
    ps.h_rowptr[r + 1] = k0 + (int)row.size();
    pd[r] = dv[o];
    pd32[r] = (float)dv[o];
    if (dir) pfix[r] = fix[o];
  }
  int st = build_halo_plan(ps.h_rowptr, ps.h_col, n, nblk, ps.plan);
  if (st != CGP_OK) return st;
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t o_perm = 0, o_rp = o_perm + al((size_t)n * 4), o_col = o_rp + al((size_t)(n + 1) * 4),
               o_k = o_col + al((size_t)nnz * 4), o_k32 = o_k + al((size_t)nnz * 8), o_d = o_k32 + al((size_t)nnz * 4),
               o_d32 = o_d + al((size_t)n * 8), o_b = o_d32 + al((size_t)n * 4), o_x = o_b + al((size_t)n * 8),
               o_f = o_x + al((size_t)n * 8), bytes = o_f + al((size_t)n);
  cudaError_t e = cudaMalloc(&ps.base, bytes);
  if (e != cudaSuccess) {
    cudaFree(ps.plan.base);
    return cuda_fail(e, "cudaMalloc(permuted system)");
  }
  char* b = static_cast<char*>(ps.base);
  ps.perm = (int*)(b + o_perm);
  ps.rowptr = (int*)(b + o_rp);
  ps.col = (int*)(b + o_col);
  ps.K = (double*)(b + o_k);
  ps.K32 = (float*)(b + o_k32);
  ps.dinv = (double*)(b + o_d);
  ps.dinv32 = (float*)(b + o_d32);
  ps.bbuf = (double*)(b + o_b);
  ps.xbuf = (double*)(b + o_x);
  ps.fixed = dir ? (unsigned char*)(b + o_f) : nullptr;
  if (e == cudaSuccess) e = cudaMemcpy(ps.perm, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ps.rowptr, ps.h_rowptr.data(), (size_t)(n + 1) * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ps.col, ps.h_col.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ps.K, pk.data(), (size_t)nnz * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ps.K32, pk32.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ps.dinv, pd.data(), (size_t)n * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ps.dinv32, pd32.data(), (size_t)n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && dir) e = cudaMemcpy(ps.fixed, pfix.data(), (size_t)n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(ps.base);
    cudaFree(ps.plan.base);
    return cuda_fail(e, "cudaMemcpy(permuted system)");
  }
  m->psys.push_back(ps);
  out = &m->psys.back();
  return CGP_OK;
}

// Solver variants of one launch.
enum SolverKind { KIND_FP64_CLASSIC = 0, KIND_MIXED = 1, KIND_FP64_SR = 2 };

SolverKind solver_kind(bool mixed, int flags) {
  return mixed ? KIND_MIXED : ((flags & 2) ? KIND_FP64_CLASSIC : KIND_FP64_SR);
}

// Dynamic shared memory of a block that keeps its rows resident: the classic
// FP64 solver needs seven vectors, the halo buffer and an FP64 CSR slice; the
// single-reduction FP64 solver nine vectors, the halo buffer, D^-1 of the
// halo, three staging buffers of the halo and the slice; the mixed solver six
// FP32 vectors, D^-1, the halo buffer, D^-1 of the halo, three staging
// buffers and an FP32 slice.
size_t res_smem_bytes(SolverKind kind, int chunk, const HaloPlan& hp) {
  const size_t ints = 4 * ((size_t)chunk + 1 + hp.max_nnz + hp.max_halo);
  size_t s = 0;
  if (kind == KIND_MIXED)
    s = 4 * ((size_t)9 * chunk + 6 * (size_t)hp.max_halo + 2 * (size_t)hp.max_nnz + 1);
  else if (kind == KIND_FP64_CLASSIC)
    s = 8 * ((size_t)7 * chunk + hp.max_halo + hp.max_nnz) + ints;
  else
    s = 8 * ((size_t)10 * chunk + 5 * (size_t)hp.max_halo + hp.max_nnz) + ints;
  return (s + 15) / 16 * 16;
}

// Bound on the barrier epochs of one solve (the counter must stay below 2^31).
long long max_epochs(const cgp_solve_opts& o) {
  return 16LL + 4LL * (long long)std::max(o.max_it, 1) + 8LL * std::max(o.max_sweeps, 1) + 8LL * 16;
}

// Shape of a persistent launch for an n-row system.  For FP64 on a mesh the
// block's rows go to shared memory when the largest chunk, its halo and its
// CSR slice fit and the grid stays co-resident.
int plan_solve(cgp_mesh_impl* m, int device, int n, int max_blocks, const SolverTuning& tu, bool mixed,
               LaunchPlan& out, PermSystem** ps_out = nullptr) {
  const int lanes = tu.lanes > 0 ? tu.lanes : 1;
  const int block = tu.block > 0 ? tu.block : 512;
  PcgFn fn0 = pcg_kernel_for(lanes, false);
  if (!fn0) return fail(CGP_ERR_INVALID_ARG, "solver tuning: lanes must be 1, 2, 4, 8 or 32");
  if (block < 64 || block > MAX_BLOCK || block % 32 != 0 || block % lanes != 0)
    return fail(CGP_ERR_INVALID_ARG, "solver tuning: block must be a multiple of 32 in [64, 512]");
  const int cap0 = std::min(coresident_blocks(fn0, block, device), max_blocks);
  if (cap0 <= 0) return fail(CGP_ERR_CUDA, "solver: kernel cannot be resident on this device");
  const int sms = std::max(1, dev_info(device).sms);
  int nblk = tu.blocks;
  if (nblk <= 0) {
    // about 256 rows per block: the FP64 work of a row is slow on this GPU's
    // narrow FP64 pipe, and even the FP32 inner solve of MIXED runs faster
    // from shared memory on several SMs than from global memory on one
    nblk = std::min(sms, std::max(1, (n + 255) / 256));
  }
  nblk = std::max(1, std::min(nblk, std::min(cap0, n)));
  out = LaunchPlan{};
  out.fn = fn0;
  out.nblk = nblk;
  out.block = block;
  // tuning flag bit 2: rows renumbered by coordinate bisection (compact chunks, smaller halos)
  PermSystem* ps = nullptr;
  if (m && (tu.flags & 4)) {
    int st = get_perm_system(m, nblk, ps);
    if (st != CGP_OK) return st;
    out.halo = ps->plan;   // the non-resident path reads the permuted pattern directly
  }
  if (ps_out) *ps_out = ps;
  if (!m || (tu.flags & 1)) return CGP_OK;
  const int chunk = (n + nblk - 1) / nblk;
  const std::vector<int>& hrp = ps ? ps->h_rowptr : m->h_rowptr;
  // rough size check before building a plan
  const int rough_nnz = hrp[std::min(n, chunk)] - hrp[0];
  PcgFn fnr = pcg_kernel_for(lanes, true);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, (const void*)fnr) != cudaSuccess) {
    cudaGetLastError();
    return CGP_OK;
  }
  const size_t limit = (size_t)std::max(0, optin_smem(device) - (int)fa.sharedSizeBytes - 1024);
  const SolverKind kind = solver_kind(mixed, tu.flags);
  if ((size_t)chunk * (kind == KIND_FP64_SR ? 80 : 56) + (size_t)rough_nnz * 12 > limit) return CGP_OK;
  HaloPlan hp;
  if (ps) {
    hp = ps->plan;
  } else {
    int st = get_halo_plan(m, nblk, hp);
    if (st != CGP_OK) return st;
  }
  const size_t smem = res_smem_bytes(kind, chunk, hp);
  if (smem > limit) return CGP_OK;
  if (cudaFuncSetAttribute((const void*)fnr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return CGP_OK;
  }
  if (coresident_blocks(fnr, block, device, smem) < nblk) return CGP_OK;
  out.fn = fnr;
  out.smem = smem;
  out.nnz_cap = hp.max_nnz;
  out.halo_cap = hp.max_halo;
  out.res = true;
  out.halo = hp;
  return CGP_OK;
}

}  // namespace

int solver_max_blocks(int device) {
  int sms = dev_info(device).sms;
  if (sms <= 0) sms = 160;
  return sms * 32;  // upper bound on co-resident blocks of >= 64 threads
}

namespace {

// Descriptor of one system solved by `nblk` blocks (blk0 set by the caller).
Desc make_desc(cgp_mesh_impl* m, const double* b, double* x, const cgp_solve_opts& o, int nblk,
               const LaunchPlan& plan, unsigned* bar, SolveResult* res, int flags) {
  Desc d{};
  d.n = m->n_c;
  d.rowptr = m->rowptr;
  d.col = m->col;
  d.val = m->far_dirichlet ? m->Kd : m->K;
  d.val32 = m->far_dirichlet ? m->Kd32 : m->K32;
  d.dinv = m->far_dirichlet ? m->dinvd : m->dinv;
  d.dinv32 = m->far_dirichlet ? m->dinvd32 : m->dinv32;
  d.fixed = m->far_dirichlet ? m->fixed : nullptr;
  d.b = b;
  d.x = x;
  d.bp = m->bp;
  d.r = m->r;
  d.z = m->z;
  d.p = m->p;
  d.p2 = m->p2;
  d.q = m->q;
  d.pub64 = m->pub64;
  d.f32pub = m->f32pub;
  d.f32own = m->f32own;
  d.fpart = m->fpart;
  d.part = m->part;
  d.tpart = m->tpart;
  d.part_stride = m->max_blocks;
  d.bar = bar;
  d.res = res;
  d.out = nullptr;
  d.blk0 = 0;
  d.nblk = nblk;
  d.tol = o.tol;
  d.inner_tol = o.inner_tol;
  d.max_it = o.max_it;
  d.max_sweeps = o.max_sweeps;
  d.use_x0 = o.use_x0;
  d.mixed = o.precision == CGP_MIXED ? 1 : 0;
  d.classic = (flags & 2) ? 1 : 0;
  d.tagged = (flags & 8) ? 1 : 0;
  d.res_nnz_cap = plan.nnz_cap;
  d.halo_cap = plan.halo_cap;
  d.lcol = plan.halo.lcol;
  d.hptr = plan.halo.hptr;
  d.hidx = plan.halo.hidx;
  d.spin_ns = 2000000000LL;
  return d;
}

}  // namespace

namespace {
// b and x0 into the bisection order, and the solution back
__global__ void perm_gather_kernel(int n, const int* __restrict__ perm, const double* __restrict__ b,
                                   const double* __restrict__ x, int use_x0, double* __restrict__ bo,
                                   double* __restrict__ xo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int o = perm[i];
  bo[i] = b[o];
  if (use_x0) xo[i] = x[o];
}

__global__ void perm_scatter_kernel(int n, const int* __restrict__ perm, const double* __restrict__ xi,
                                    double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[perm[i]] = xi[i];
}
}  // namespace

int launch_solve(cgp_mesh_impl* m, const double* b, double* x, const cgp_solve_opts& o, cgp_solve_info* info_dev,
                 cudaStream_t s) {
  const bool mixed = o.precision == CGP_MIXED;
  const SolverTuning& tu = m->tune[mixed ? CGP_TUNE_SOLVE_MIXED : CGP_TUNE_SOLVE_FP64];
  LaunchPlan plan;
  PermSystem* ps = nullptr;
  int st = plan_solve(m, m->device, m->n_c, m->max_blocks, tu, mixed, plan, &ps);
  if (st != CGP_OK) return st;
  const int nblk = plan.nblk;
  // barrier epochs stay far below 2^32 / nblk
  if (max_epochs(o) * nblk >= (1LL << 31)) return fail(CGP_ERR_INVALID_ARG, "solver: max_it too large");

  Desc d = make_desc(m, b, x, o, nblk, plan, m->bar, m->res, tu.flags);
  d.out = info_dev;
  const int n = m->n_c;
  if (ps) {   // the same solve on the renumbered system
    d.rowptr = ps->rowptr;
    d.col = ps->col;
    d.val = ps->K;
    d.val32 = ps->K32;
    d.dinv = ps->dinv;
    d.dinv32 = ps->dinv32;
    d.fixed = ps->fixed;
    d.b = ps->bbuf;
    d.x = ps->xbuf;
    d.lcol = ps->plan.lcol;
    d.hptr = ps->plan.hptr;
    d.hidx = ps->plan.hidx;
    perm_gather_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, ps->perm, b, x, o.use_x0, ps->bbuf, ps->xbuf);
    CGP_CUDA(cudaGetLastError());
  }

  CGP_CUDA(cudaMemsetAsync(m->bar, 0, 256, s));
  CGP_CUDA(cudaMemsetAsync(m->res, 0, sizeof(SolveResult), s));
  void* args[] = {&d};
  CGP_CUDA(cudaLaunchCooperativeKernel((const void*)plan.fn, dim3(nblk), dim3(plan.block), args, plan.smem, s));
  if (ps) {
    perm_scatter_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, ps->perm, ps->xbuf, x);
    CGP_CUDA(cudaGetLastError());
  }
  m->last_plan[mixed ? 1 : 0] = PlanRecord{nblk, plan.block, plan.res ? 1 : 0, (int)plan.smem};
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
  LaunchPlan plan;
  const SolverTuning tu{0, 1, 0, 3};   // default shape, vectors in global scratch, classic FP64 iteration
  int st = plan_solve(nullptr, device, sys.n, scr.max_blocks, tu, false, plan);
  if (st != CGP_OK) return st;
  const int nblk = plan.nblk;
  if (max_epochs(o) * nblk >= (1LL << 31)) return fail(CGP_ERR_INVALID_ARG, "solver: max_it too large");
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
  d.p2 = scr.p2;
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
  d.classic = 1;
  d.res_nnz_cap = 0;
  d.spin_ns = 2000000000LL;
  void* args[] = {&d};
  CGP_CUDA(cudaLaunchCooperativeKernel((const void*)plan.fn, dim3(nblk), dim3(plan.block), args, 0, s));
  return CGP_OK;
}

int launch_spmv(cgp_mesh_impl* m, int precision, const void* x, void* y, cudaStream_t s) {
  const int sms = std::max(1, dev_info(m->device).sms);
  const SolverTuning& tu = m->tune[precision == CGP_FP64 ? CGP_TUNE_SPMV_FP64 : CGP_TUNE_SPMV_FP32];
  if (tu.flags & 1) return launch_spmv_stencil(m, precision, x, y, tu.block, s);   // O-grid stencil form
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

// ---------------------------------------------------------------------------
// Batched solves: many meshes, one persistent cooperative launch
// ---------------------------------------------------------------------------
struct BatchShape {
  int block = 512;
  int lanes = 1;
  int per_sm = 0;   // blocks per SM (0: as many as can be co-resident)
  int flags = 0;    // bit 0: rows in global memory; bit 1: classic FP64 iteration; bit 2: one packed launch
};

}  // namespace cgp

struct cgp_batch_s {
  int device = 0;
  int count = 0;
  std::vector<cgp::cgp_mesh_impl*> meshes;
  std::vector<const double*> b;
  std::vector<double*> x;
  cgp_solve_opts opts{};
  cgp::BatchShape shape;
  // plan
  int grid = 0;
  bool res = false;
  size_t smem = 0;
  cgp::BatchFn fn = nullptr;
  std::vector<int> nblk;
  // waves: cooperative launches run one after the other, each over a subset of
  // the instances (one wave holding all of them when packed)
  struct Wave {
    int grid;
    int blk_off;    // offset of its block -> instance map
    bool res;
    size_t smem;
    cgp::BatchFn fn;
  };
  std::vector<Wave> waves;
  // device buffers: descriptors, block -> instance map, control area
  void* d_desc = nullptr;
  int* d_blk_inst = nullptr;
  unsigned char* d_ctrl = nullptr;   // per instance: barrier (256 B) + result (256 B); then t_start
  size_t ctrl_bytes = 0;
};

namespace cgp {
namespace {

constexpr size_t kCtrlPerInstance = 512;

int batch_plan(cgp_batch_s* B, const BatchShape& sh, const cgp_solve_opts& o) {
  const int lanes = sh.lanes > 0 ? sh.lanes : 1;
  const int block = sh.block > 0 ? sh.block : 512;
  const bool mixed = o.precision == CGP_MIXED;
  BatchFn fn0 = batched_kernel_for(lanes, false);
  if (!fn0 || block < 64 || block > MAX_BLOCK || block % 32 != 0 || block % lanes != 0)
    return fail(CGP_ERR_INVALID_ARG, "batch tuning: bad block or lanes");
  const int sms = std::max(1, dev_info(B->device).sms);
  int per_sm0 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm0, (const void*)fn0, block, 0) != cudaSuccess) {
    cudaGetLastError();
    return fail(CGP_ERR_CUDA, "batch: occupancy query failed");
  }
  int G = per_sm0 * sms;
  if (sh.per_sm > 0) G = std::min(G, sh.per_sm * sms);
  const int count = B->count;
  if (G < count) return fail(CGP_ERR_INVALID_ARG, "batch: more instances than co-resident blocks");
  // blocks per instance in proportion to nnz * sqrt(n) (work of a CG solve on a 2-D mesh)
  std::vector<double> w(count);
  double W = 0.0;
  for (int i = 0; i < count; ++i) {
    w[i] = (double)B->meshes[i]->nnz * std::sqrt((double)B->meshes[i]->n_c);
    W += w[i];
  }
  std::vector<int> nb(count), cap(count);
  int total = 0;
  for (int i = 0; i < count; ++i) {
    cap[i] = std::max(1, std::min(B->meshes[i]->n_c / 64, B->meshes[i]->max_blocks));
    nb[i] = std::max(1, std::min(cap[i], (int)std::floor(G * w[i] / W)));
    total += nb[i];
  }
  while (total > G) {  // shrink the instance with the most blocks
    int j = (int)(std::max_element(nb.begin(), nb.end()) - nb.begin());
    if (nb[j] <= 1) break;
    --nb[j];
    --total;
  }
  while (total < G) {  // grow the instance with the most work per block
    int j = -1;
    double best = 0.0;
    for (int i = 0; i < count; ++i)
      if (nb[i] < cap[i] && w[i] / nb[i] > best) {
        best = w[i] / nb[i];
        j = i;
      }
    if (j < 0) break;
    ++nb[j];
    ++total;
  }
  // shared-memory residency when every instance's chunk fits
  std::vector<HaloPlan> hp(count);
  const SolverKind kind = solver_kind(mixed, sh.flags);
  bool res = !(sh.flags & 1);
  size_t smem = 0;
  BatchFn fnr = batched_kernel_for(lanes, true);
  cudaFuncAttributes fa{};
  if (res && cudaFuncGetAttributes(&fa, (const void*)fnr) != cudaSuccess) {
    cudaGetLastError();
    res = false;
  }
  const size_t limit = res ? (size_t)std::max(0, optin_smem(B->device) - (int)fa.sharedSizeBytes - 1024) : 0;
  for (int i = 0; res && i < count; ++i) {
    cgp_mesh_impl* m = B->meshes[i];
    const int chunk = (m->n_c + nb[i] - 1) / nb[i];
    const int rough_nnz = m->h_rowptr[std::min(m->n_c, chunk)] - m->h_rowptr[0];
    if ((size_t)chunk * (kind == KIND_FP64_SR ? 80 : 56) + (size_t)rough_nnz * 12 > limit) {
      res = false;
      break;
    }
    int st = get_halo_plan(m, nb[i], hp[i]);
    if (st != CGP_OK) return st;
    smem = std::max(smem, res_smem_bytes(kind, chunk, hp[i]));
    if (smem > limit) res = false;
  }
  if (res) {
    if (cudaFuncSetAttribute((const void*)fnr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      res = false;
    } else {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fnr, block, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
      }
      if (per_sm * sms < total) res = false;
    }
  }
  if (!res) smem = 0;
  B->waves.assign(1, cgp_batch_s::Wave{total, 0, res, smem, res ? fnr : fn0});
  // descriptors
  std::vector<Desc> desc(count);
  std::vector<int> blk_inst(total);
  int blk0 = 0;
  for (int i = 0; i < count; ++i) {
    cgp_mesh_impl* m = B->meshes[i];
    LaunchPlan lp;
    lp.nblk = nb[i];
    lp.block = block;
    if (res) {
      lp.res = true;
      lp.nnz_cap = hp[i].max_nnz;
      lp.halo_cap = hp[i].max_halo;
      lp.halo = hp[i];
    }
    unsigned char* ctrl = B->d_ctrl + kCtrlPerInstance * i;
    desc[i] = make_desc(m, B->b[i], B->x[i], o, nb[i], lp, reinterpret_cast<unsigned*>(ctrl),
                        reinterpret_cast<SolveResult*>(ctrl + 256), sh.flags);
    desc[i].blk0 = blk0;
    if (max_epochs(o) * nb[i] >= (1LL << 31)) return fail(CGP_ERR_INVALID_ARG, "batch: max_it too large");
    for (int k = 0; k < nb[i]; ++k) blk_inst[blk0 + k] = i;
    blk0 += nb[i];
  }
  CGP_CUDA(cudaMemcpy(B->d_desc, desc.data(), sizeof(Desc) * count, cudaMemcpyHostToDevice));
  CGP_CUDA(cudaMemcpy(B->d_blk_inst, blk_inst.data(), sizeof(int) * total, cudaMemcpyHostToDevice));
  B->grid = total;
  B->res = res;
  B->smem = smem;
  B->fn = res ? fnr : fn0;
  B->nblk = nb;
  B->shape = BatchShape{block, lanes, sh.per_sm, sh.flags};
  return CGP_OK;
}

// Wave schedule: every instance gets the block count a solve of it alone
// would use (about 256 rows per block, at most one SM's worth of blocks
// each), so that it can keep its rows in shared memory; instances are packed
// largest first into waves of at most blocks_per_sm x SMs blocks, and the
// waves run as consecutive cooperative launches.  Small instances then share
// the GPU while each large one gets all of it.
int batch_plan_waves(cgp_batch_s* B, const BatchShape& sh, const cgp_solve_opts& o) {
  const int lanes = sh.lanes > 0 ? sh.lanes : 1;
  const int block = sh.block > 0 ? sh.block : 512;
  const bool mixed = o.precision == CGP_MIXED;
  BatchFn fn0 = batched_kernel_for(lanes, false), fnr = batched_kernel_for(lanes, true);
  if (!fn0 || block < 64 || block > MAX_BLOCK || block % 32 != 0 || block % lanes != 0)
    return fail(CGP_ERR_INVALID_ARG, "batch tuning: bad block or lanes");
  const int sms = std::max(1, dev_info(B->device).sms);
  // blocks of this size that fit on one SM with rows in global memory: a wave
  // never asks for more than that, whatever blocks_per_sm requests
  int fit = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, (const void*)fn0, block, 0) != cudaSuccess || fit < 1) {
    cudaGetLastError();
    return fail(CGP_ERR_CUDA, "batch: occupancy query failed");
  }
  const int cap = sms * std::min(std::max(1, sh.per_sm), fit);
  const int count = B->count;
  const SolverKind kind = solver_kind(mixed, sh.flags);
  std::vector<int> nb(count), order(count);
  for (int i = 0; i < count; ++i) {
    const int n = B->meshes[i]->n_c;
    nb[i] = std::max(1, std::min(std::min(cap, B->meshes[i]->max_blocks), (n + 255) / 256));
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nb[a] > nb[b]; });
  std::vector<std::vector<int>> groups;
  std::vector<int> used;
  for (int i : order) {
    size_t g = 0;
    while (g < groups.size() && used[g] + nb[i] > cap) ++g;
    if (g == groups.size()) {
      groups.emplace_back();
      used.push_back(0);
    }
    groups[g].push_back(i);
    used[g] += nb[i];
  }
  cudaFuncAttributes fa{};
  bool can_res = !(sh.flags & 1) && cudaFuncGetAttributes(&fa, (const void*)fnr) == cudaSuccess;
  if (!can_res) cudaGetLastError();
  const size_t limit = can_res ? (size_t)std::max(0, optin_smem(B->device) - (int)fa.sharedSizeBytes - 1024) : 0;
  std::vector<Desc> desc(count);
  std::vector<int> blk_inst;
  std::vector<cgp_batch_s::Wave> waves;
  size_t max_smem = 0;
  for (const auto& grp : groups) {
    int total = 0;
    for (int i : grp) total += nb[i];
    bool res = can_res;
    size_t smem = 0;
    std::vector<HaloPlan> hp(count);
    for (int i : grp) {
      if (!res) break;
      cgp_mesh_impl* m = B->meshes[i];
      const int chunk = (m->n_c + nb[i] - 1) / nb[i];
      const int rough_nnz = m->h_rowptr[std::min(m->n_c, chunk)] - m->h_rowptr[0];
      if ((size_t)chunk * (kind == KIND_FP64_SR ? 80 : 56) + (size_t)rough_nnz * 12 > limit) {
        res = false;
        break;
      }
      int st = get_halo_plan(m, nb[i], hp[i]);
      if (st != CGP_OK) return st;
      smem = std::max(smem, res_smem_bytes(kind, chunk, hp[i]));
      if (smem > limit) res = false;
    }
    if (res) {
      int per_sm = 0;
      if (cudaFuncSetAttribute((const void*)fnr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)std::max(smem, max_smem)) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fnr, block, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
      }
      if (per_sm * sms < total) res = false;
    }
    if (!res) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn0, block, 0) != cudaSuccess) {
        cudaGetLastError();
        return fail(CGP_ERR_CUDA, "batch: occupancy query failed");
      }
      if (per_sm * sms < total) return fail(CGP_ERR_INVALID_ARG, "batch: a wave does not fit the device");
      smem = 0;
    }
    max_smem = std::max(max_smem, smem);
    const int off = (int)blk_inst.size();
    int blk0 = 0;
    for (int i : grp) {
      cgp_mesh_impl* m = B->meshes[i];
      LaunchPlan lp;
      lp.nblk = nb[i];
      lp.block = block;
      if (res) {
        lp.res = true;
        lp.nnz_cap = hp[i].max_nnz;
        lp.halo_cap = hp[i].max_halo;
        lp.halo = hp[i];
      }
      unsigned char* ctrl = B->d_ctrl + kCtrlPerInstance * i;
      desc[i] = make_desc(m, B->b[i], B->x[i], o, nb[i], lp, reinterpret_cast<unsigned*>(ctrl),
                          reinterpret_cast<SolveResult*>(ctrl + 256), sh.flags);
      desc[i].blk0 = blk0;
      if (max_epochs(o) * nb[i] >= (1LL << 31)) return fail(CGP_ERR_INVALID_ARG, "batch: max_it too large");
      for (int k = 0; k < nb[i]; ++k) blk_inst.push_back(i);
      blk0 += nb[i];
    }
    waves.push_back(cgp_batch_s::Wave{total, off, res, smem, res ? fnr : fn0});
  }
  if (blk_inst.size() > (size_t)sms * std::max(32, count)) return fail(CGP_ERR_INVALID_ARG, "batch: too many blocks");
  CGP_CUDA(cudaMemcpy(B->d_desc, desc.data(), sizeof(Desc) * count, cudaMemcpyHostToDevice));
  CGP_CUDA(cudaMemcpy(B->d_blk_inst, blk_inst.data(), sizeof(int) * blk_inst.size(), cudaMemcpyHostToDevice));
  B->waves = waves;
  B->grid = 0;
  B->res = true;
  for (const auto& w : waves) {
    B->grid = std::max(B->grid, w.grid);
    B->res = B->res && w.res;
  }
  B->smem = max_smem;
  B->fn = waves[0].fn;
  B->nblk = nb;
  B->shape = BatchShape{block, lanes, sh.per_sm, sh.flags};
  return CGP_OK;
}

int batch_plan_any(cgp_batch_s* B, const BatchShape& sh, const cgp_solve_opts& o) {
  return (sh.flags & 4) ? batch_plan(B, sh, o) : batch_plan_waves(B, sh, o);
}

int batch_launch(cgp_batch_s* B, cudaStream_t s) {
  CGP_CUDA(cudaMemsetAsync(B->d_ctrl, 0, B->ctrl_bytes, s));
  unsigned long long* t_start = reinterpret_cast<unsigned long long*>(B->d_ctrl + kCtrlPerInstance * B->count);
  const Desc* descs = static_cast<const Desc*>(B->d_desc);
  for (size_t w = 0; w < B->waves.size(); ++w) {
    const int* bi = B->d_blk_inst + B->waves[w].blk_off;
    unsigned long long* ts = w == 0 ? t_start : nullptr;   // the batch starts with its first wave
    void* args[] = {&descs, &bi, &ts};
    CGP_CUDA(cudaLaunchCooperativeKernel((const void*)B->waves[w].fn, dim3(B->waves[w].grid),
                                         dim3(B->shape.block), args, B->waves[w].smem, s));
  }
  return CGP_OK;
}

}  // namespace

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

static bool valid_shape(int what, int block, int lanes) {
  const int max_block = (what == CGP_TUNE_SOLVE_FP64 || what == CGP_TUNE_SOLVE_MIXED) ? MAX_BLOCK : 256;
  if (block != 0 && (block < 64 || block > max_block || block % 32 != 0)) return false;
  if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 32) return false;
  return true;
}

extern "C" int cgp_set_tuning(cgp_mesh m, int what, int block, int lanes, int blocks, int flags) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_set_tuning: NULL mesh");
  if (what < 0 || what > 3) return fail(CGP_ERR_INVALID_ARG, "cgp_set_tuning: unknown target");
  if (!valid_shape(what, block, lanes) || blocks < 0 || (flags & ~15))
    return fail(CGP_ERR_INVALID_ARG, "cgp_set_tuning: block must be 0 or a multiple of 32 in [64, 512] "
                                     "(solver) or [64, 256] (SpMV), "
                                     "lanes 0, 1, 2, 4, 8 or 32, blocks >= 0, flags 0 to 15");
  m->tune[what] = SolverTuning{block, lanes, blocks, flags};
  return CGP_OK;
}

extern "C" int cgp_get_tuning(cgp_mesh m, int what, int* block, int* lanes, int* blocks, int* flags) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_get_tuning: NULL mesh");
  if (what < 0 || what > 3) return fail(CGP_ERR_INVALID_ARG, "cgp_get_tuning: unknown target");
  if (block) *block = m->tune[what].block;
  if (lanes) *lanes = m->tune[what].lanes;
  if (blocks) *blocks = m->tune[what].blocks;
  if (flags) *flags = m->tune[what].flags;
  return CGP_OK;
}

extern "C" int cgp_last_launch(cgp_mesh m, int precision, int* blocks, int* block, int* resident,
                               int* smem_bytes) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_last_launch: NULL mesh");
  if (precision != CGP_FP64 && precision != CGP_MIXED) return fail(CGP_ERR_INVALID_ARG, "cgp_last_launch: precision");
  const PlanRecord& r = m->last_plan[precision == CGP_MIXED ? 1 : 0];
  if (blocks) *blocks = r.blocks;
  if (block) *block = r.block;
  if (resident) *resident = r.resident;
  if (smem_bytes) *smem_bytes = r.smem;
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

// ---------------------------------------------------------------------------
// batch C ABI
// ---------------------------------------------------------------------------
extern "C" int cgp_batch_create(const cgp_mesh* meshes, int count, const double* const* b, double* const* x,
                                const cgp_solve_opts* opts, cgp_batch* out) {
  if (!out) return fail(CGP_ERR_INVALID_ARG, "cgp_batch_create: out is NULL");
  *out = nullptr;
  if (!meshes || !b || !x || count < 1) return fail(CGP_ERR_INVALID_ARG, "cgp_batch_create: bad arguments");
  cgp_solve_opts o;
  for (int i = 0; i < count; ++i) {
    if (!meshes[i] || !b[i] || !x[i]) return fail(CGP_ERR_INVALID_ARG, "cgp_batch_create: NULL entry");
    for (int j = 0; j < i; ++j)
      if (meshes[j] == meshes[i])
        return fail(CGP_ERR_INVALID_ARG, "cgp_batch_create: a mesh appears twice (its scratch would be shared)");
  }
  int st = check_solve_args(meshes[0], b[0], x[0], opts, o);
  if (st != CGP_OK) return st;
  cgp_batch_s* B = new cgp_batch_s();
  B->count = count;
  B->opts = o;
  cudaError_t e = cudaGetDevice(&B->device);
  if (e != cudaSuccess) {
    delete B;
    return cuda_fail(e, "cudaGetDevice");
  }
  for (int i = 0; i < count; ++i) {
    B->meshes.push_back(meshes[i]);
    B->b.push_back(b[i]);
    B->x.push_back(x[i]);
  }
  B->ctrl_bytes = kCtrlPerInstance * count + 256;
  const int sms = std::max(1, dev_info(B->device).sms);
  const size_t max_grid = (size_t)sms * std::max(32, count);   // waves: up to one SM's worth of blocks per instance
  e = cudaMalloc(&B->d_desc, sizeof(Desc) * count);
  if (e == cudaSuccess) e = cudaMalloc(&B->d_blk_inst, sizeof(int) * max_grid);
  if (e == cudaSuccess) e = cudaMalloc(&B->d_ctrl, B->ctrl_bytes);
  if (e != cudaSuccess) {
    cgp_batch_destroy(B);
    return cuda_fail(e, "cudaMalloc(batch)");
  }
  st = batch_plan_any(B, BatchShape{}, o);
  if (st != CGP_OK) {
    cgp_batch_destroy(B);
    return st;
  }
  *out = B;
  return CGP_OK;
}

extern "C" int cgp_batch_set_tuning(cgp_batch batch, int block, int lanes, int blocks_per_sm, int flags) {
  if (!batch) return fail(CGP_ERR_INVALID_ARG, "cgp_batch_set_tuning: NULL batch");
  if (!valid_shape(CGP_TUNE_SOLVE_FP64, block, lanes) || blocks_per_sm < 0 || (flags & ~15))
    return fail(CGP_ERR_INVALID_ARG, "cgp_batch_set_tuning: bad shape");
  return batch_plan_any(batch, BatchShape{block, lanes, blocks_per_sm, flags}, batch->opts);
}

extern "C" int cgp_batch_solve(cgp_batch batch, void* stream) {
  if (!batch) return fail(CGP_ERR_INVALID_ARG, "cgp_batch_solve: NULL batch");
  return batch_launch(batch, (cudaStream_t)stream);
}

extern "C" int cgp_batch_info(cgp_batch batch, cgp_solve_info* infos, double* seconds) {
  if (!batch) return fail(CGP_ERR_INVALID_ARG, "cgp_batch_info: NULL batch");
  std::vector<unsigned char> h(batch->ctrl_bytes);
  CGP_CUDA(cudaDeviceSynchronize());
  CGP_CUDA(cudaMemcpy(h.data(), batch->d_ctrl, batch->ctrl_bytes, cudaMemcpyDeviceToHost));
  unsigned long long t0 = 0;
  std::memcpy(&t0, h.data() + kCtrlPerInstance * batch->count, sizeof(t0));
  int worst = CGP_OK;
  for (int i = 0; i < batch->count; ++i) {
    SolveResult r;
    std::memcpy(&r, h.data() + kCtrlPerInstance * i + 256, sizeof(r));
    const int status = r.timeout ? CGP_ERR_TIMEOUT : r.status;
    if (infos) {
      infos[i].iterations = r.iterations;
      infos[i].outer_sweeps = r.sweeps;
      infos[i].rel_res_recursive = r.rel_rec;
      infos[i].rel_res_true = r.rel_true;
      infos[i].status = status;
    }
    if (seconds) seconds[i] = r.t_end > t0 ? (double)(r.t_end - t0) * 1e-9 : 0.0;
    if (status != CGP_OK && worst == CGP_OK) worst = status;
  }
  if (worst != CGP_OK) return fail(worst, "cgp_batch_info: at least one instance did not converge");
  return CGP_OK;
}

extern "C" int cgp_batch_query(cgp_batch batch, int* grid, int* block, int* lanes, int* resident, int* blocks) {
  if (!batch) return fail(CGP_ERR_INVALID_ARG, "cgp_batch_query: NULL batch");
  if (grid) *grid = batch->grid;
  if (block) *block = batch->shape.block;
  if (lanes) *lanes = batch->shape.lanes;
  if (resident) *resident = batch->res ? 1 : 0;
  if (blocks)
    for (int i = 0; i < batch->count; ++i) blocks[i] = batch->nblk[i];
  return CGP_OK;
}

extern "C" int cgp_batch_autotune(cgp_batch batch, void* stream, double* best_ms) {
  if (!batch) return fail(CGP_ERR_INVALID_ARG, "cgp_batch_autotune: NULL batch");
  cudaStream_t s = (cudaStream_t)stream;
  cgp_solve_opts o = batch->opts;
  o.use_x0 = 0;  // every candidate solves the same problem from zero
  cudaEvent_t e0, e1;
  CGP_CUDA(cudaEventCreate(&e0));
  CGP_CUDA(cudaEventCreate(&e1));
  BatchShape best{};
  float best_t = 1e30f;
  const int blocks[2] = {256, 512};
  const int lanes[2] = {1, 2};
  const int per_sm[2] = {1, 2};
  const int nflags = batch->opts.precision == CGP_MIXED ? 2 : 4;
  for (int fl = 0; fl < 2 * nflags; ++fl)   // bit 2 (one packed launch instead of waves) on top
    for (int bk : blocks)
      for (int ln : lanes)
        for (int ps : per_sm) {
          BatchShape cand{bk, ln, ps, (fl % nflags) | (fl >= nflags ? 4 : 0)};
          if (batch_plan_any(batch, cand, o) != CGP_OK) continue;
          float t = 1e30f;
          for (int rep = 0; rep < 2; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess || batch_launch(batch, s) != CGP_OK ||
                cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
              break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, ms);
          }
          if (t < best_t) {
            best_t = t;
            best = cand;
          }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_t >= 1e29f) return fail(CGP_ERR_CUDA, "cgp_batch_autotune: no candidate ran");
  int st = batch_plan_any(batch, best, batch->opts);
  if (st != CGP_OK) return st;
  if (best_ms) *best_ms = best_t;
  return CGP_OK;
}

extern "C" int cgp_batch_destroy(cgp_batch batch) {
  if (!batch) return fail(CGP_ERR_INVALID_ARG, "cgp_batch_destroy: NULL batch");
  cudaDeviceSynchronize();
  if (batch->d_desc) cudaFree(batch->d_desc);
  if (batch->d_blk_inst) cudaFree(batch->d_blk_inst);
  if (batch->d_ctrl) cudaFree(batch->d_ctrl);
  delete batch;
  return CGP_OK;
}

extern "C" int cgp_poisson_solve_batched(const cgp_mesh* meshes, int count, const double* const* b,
                                         double* const* x, const cgp_solve_opts* opts, cgp_solve_info* infos,
                                         void* stream) {
  cgp_batch batch = nullptr;
  int st = cgp_batch_create(meshes, count, b, x, opts, &batch);
  if (st != CGP_OK) return st;
  st = cgp_batch_solve(batch, stream);
  if (st == CGP_OK && infos) st = cgp_batch_info(batch, infos, nullptr);
  if (st == CGP_OK && !infos) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
  }
  const std::string msg = cgp_last_error();
  cgp_batch_destroy(batch);
  if (st != CGP_OK) fail(st, msg);
  return st;
}

// ---------------------------------------------------------------------------
// autotuner for single solves
// ---------------------------------------------------------------------------
namespace {

std::string device_name(int device) {
  cudaDeviceProp p{};
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string n = p.name;
  for (char& c : n)
    if (c == ' ') c = '_';
  return n;
}

// Cache lines: "<gpu> <n> <nnz> <target> <block> <lanes> <blocks> <flags> <ms>"
bool cache_lookup(const char* path, const std::string& gpu, int n, int nnz, int what, SolverTuning& out) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char name[256];
  int cn, cnnz, cw, b, l, k, fl;
  double ms;
  bool found = false;
  while (std::fscanf(f, "%255s %d %d %d %d %d %d %d %lf", name, &cn, &cnnz, &cw, &b, &l, &k, &fl, &ms) == 9) {
    if (gpu == name && cn == n && cnnz == nnz && cw == what) {
      out = SolverTuning{b, l, k, fl};
      found = true;  // the last matching line wins
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& gpu, int n, int nnz, int what, const SolverTuning& t,
                 double ms) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d %d %d %d %.6f\n", gpu.c_str(), n, nnz, what, t.block, t.lanes, t.blocks,
               t.flags, ms);
  std::fclose(f);
}

}  // namespace

extern "C" int cgp_autotune(cgp_mesh m, int precision, const double* b, double* x, const char* cache_path,
                            void* stream, double* best_ms) {
  if (!m || !b || !x) return fail(CGP_ERR_INVALID_ARG, "cgp_autotune: NULL argument");
  if (precision != CGP_FP64 && precision != CGP_MIXED) return fail(CGP_ERR_INVALID_ARG, "cgp_autotune: precision");
  const int what = precision == CGP_MIXED ? CGP_TUNE_SOLVE_MIXED : CGP_TUNE_SOLVE_FP64;
  const std::string gpu = device_name(m->device);
  SolverTuning cached{};
  if (cache_lookup(cache_path, gpu, m->n_c, m->nnz, what, cached)) {
    m->tune[what] = cached;
    if (best_ms) *best_ms = -1.0;
    return CGP_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cgp_solve_opts o{1e-8, 20000, precision, 1e-4, 0, 50};
  const int sms = std::max(1, dev_info(m->device).sms);
  std::vector<int> counts;
  if (m->n_c <= 16384) counts = {1, 2, 4, 8, 16};
  for (int c : {sms / 2, sms, 2 * sms})
    if (c >= 1 && c <= m->n_c / 32) counts.push_back(c);
  if (counts.empty()) counts.push_back(1);
  cudaEvent_t e0, e1;
  CGP_CUDA(cudaEventCreate(&e0));
  CGP_CUDA(cudaEventCreate(&e1));
  const SolverTuning saved = m->tune[what];
  SolverTuning best{};
  float best_t = 1e30f;
  // bit 1 (classic FP64 iteration) and bit 3 (tagged reductions of the
  // single-reduction form) only for FP64; bit 2 (bisection order) for both
  std::vector<int> flag_set;
  for (int fl = 0; fl < 16; ++fl) {
    if (precision == CGP_MIXED && (fl & 10)) continue;
    if ((fl & 2) && (fl & 8)) continue;
    flag_set.push_back(fl);
  }
  for (int fl : flag_set)
    for (int bk : {256, 512})
      for (int ln : {1, 2, 4})
        for (int c : counts) {
          m->tune[what] = SolverTuning{bk, ln, c, fl};
          float t = 1e30f;
          for (int rep = 0; rep < 2; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess || launch_solve(m, b, x, o, nullptr, s) != CGP_OK ||
                cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
              break;
            // only a candidate that converged counts
            SolveResult r{};
            if (cudaMemcpy(&r, m->res, sizeof(SolveResult), cudaMemcpyDeviceToHost) != cudaSuccess ||
                r.timeout || r.status != CGP_OK)
              break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, ms);
          }
          cudaGetLastError();
          if (t < best_t) {
            best_t = t;
            best = m->tune[what];
          }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_t >= 1e29f) {
    m->tune[what] = saved;
    return fail(CGP_ERR_CUDA, "cgp_autotune: no candidate ran");
  }
  m->tune[what] = best;
  cache_store(cache_path, gpu, m->n_c, m->nnz, what, best, best_t);
  if (best_ms) *best_ms = best_t;
  return CGP_OK;
}
