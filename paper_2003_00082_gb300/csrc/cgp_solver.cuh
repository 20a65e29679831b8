// Device side of the persistent Jacobi-PCG solver (Eqs. 12, 15): the
// per-launch descriptor, block-group barriers, exact fixed-point grid
// reductions (plain and tagged slots), the CSR products over a block's rows,
// and the FP64 (textbook and single-reduction) and mixed-precision solve
// loops.  Included by every translation unit that instantiates solver
// kernels; everything here has internal linkage, so each unit compiles its
// own copy of what it uses.
#pragma once

#include <cmath>

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
  double* pub64;      // FP64 published vectors: single-reduction R[2], W[2], S[2] ([6][n] doubles);
                      // pipelined tagged W[3], Z[3], N[3] ([9][n] 16-byte words)
  float* f32pub;      // mixed: published R[2], W[2], S[2] ([6][n])
  float* f32own;      // mixed without RES: own r, u, w, p, s, e ([6][n])
  float* fpart;       // mixed: FP32 partial slots [2][NCOMP][part_stride]
  double* part;
  unsigned long long* tpart;  // FP64 single-reduction: tagged slots [2][3][part_stride] (128-bit)
  unsigned* nflag;    // FP64 pipelined tiles: per block, the count of its published w (release)
  int part_stride;
  unsigned* bar;
  SolveResult* res;
  cgp_solve_info* out;  // optional device copy of the outcome
  int blk0, nblk;
  double tol, inner_tol;
  int max_it, max_sweeps, use_x0, mixed;
  int classic;        // FP64: two barriers per iteration (Saad, Alg. 9.1) instead of the single-reduction form
  int tagged;         // FP64 single-reduction: reductions through tagged slots instead of the group barrier
  int pipelined;      // FP64: pipelined iteration (CSR: kernels of cgp_pipe.cu; tiles: solve_fp64_pl; rows resident only)
  int stencil;        // FP64, rows resident: O-grid tiles with the seven-point stencil product
  int box_cap;        // stencil: doubles of a block's padded box
  const double* planes;  // stencil: [7][n] coefficients (offsets as in stencil_offset)
  const int* bpos;    // stencil: [n] box position of every row
  const int* bdim;    // stencil: [nblk] box row length
  const int* hpos;    // stencil: box position of every halo entry (lists by d.hptr / d.hidx)
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

// Tests of a double on its bits (integer instructions).
__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7FF) != 0x7FF;
}
__device__ __forceinline__ bool positive_bits(double x) { return __double_as_longlong(x) > 0; }   // > +0 or NaN
__device__ __forceinline__ bool nonneg_le(double x, double y) {   // x <= y for x, y >= 0
  return __double_as_longlong(x) <= __double_as_longlong(y);
}

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
// (red & 1) of d.part.  The sums are exact fixed-point integer sums
// (cgp_fixed.h): they run on the integer pipe, cost no FP64 instructions, and
// do not depend on the order of the terms.
template <int NC>
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
      ulonglong2* slot = reinterpret_cast<ulonglong2*>(part_slot(d, red, c, lb));
      slot[0] = make_ulonglong2((unsigned long long)x, (unsigned long long)(x >> 64));
      slot[1] = make_ulonglong2((unsigned long long)E, 0ull);
    }
  }
}

// ---- 64-bit fixed-point block sums ------------------------------------------
// Relative to a reference exponent E >= e, a finite double v = M 2^(e - 1075)
// (M < 2^53 with the implicit bit; e = 1 for zero and subnormals) has the
// image X = (M << 4) >> (E - e) = v 2^(1079 - E) truncated, |X| < 2^57.  A
// warp adds its images exactly in three 26/26/12-bit limbs with redux.sync.
// The sums are deterministic (fixed assignment of rows to threads and of
// threads to warps) and exact up to the truncation of each term 2^-54 below
// the largest one of its warp or block.
__device__ __forceinline__ int fx64_exponent(double v) { return fx::exponent_of(v); }
__device__ __forceinline__ long long fx64_image(double v, int E) { return (long long)fx::image64(v, E); }

// exact warp sum of |x| < 2^57 per lane (|sum| < 2^62), on every lane
__device__ __forceinline__ long long warp_sum57(long long x) {
  const unsigned s0 = __reduce_add_sync(0xffffffffu, (unsigned)(x & 0x3FFFFFF));
  const unsigned s1 = __reduce_add_sync(0xffffffffu, (unsigned)((x >> 26) & 0x3FFFFFF));
  const int s2 = __reduce_add_sync(0xffffffffu, (int)(x >> 52));
  return (long long)s0 + ((long long)s1 << 26) + ((long long)s2 << 52);
}

// Tagged slot of a 64-bit block partial S (|S| < 2^62, value S 2^(E - 1074)):
// the layout of fx::pack_tagged with S stored unshifted, read back by
// tagged_total<kSlot64Shift>.
constexpr int kSlot64Shift = 55;
__device__ __forceinline__ void store_slot64(ulonglong2* slot, long long S, int E, int red) {
  uint64_t lo, hi;
  fx::pack_tagged((fx::I128)S, E, red, lo, hi, 0);
  st_relaxed_b128(slot, lo, hi);
}

// Tagged reductions with 64-bit fixed-point partials: every warp sums its
// lanes' values exactly in REDUX limbs (fx64_image relative to the warp's
// largest exponent), warp c folds the block's warp sums of component c
// (aligned to the block's largest exponent, 5 bits of headroom for up to 32
// warps) and stores the block's partial in its tagged slot (store_slot64;
// read back by tagged_total<kSlot64Shift>).  Deterministic, and exact up to
// the truncation of each term 2^-54 below the largest one of its warp or
// block: far fewer integer instructions than the 128-bit sums of
// put_partials, which the untagged reductions keep.
template <int NC>
__device__ __forceinline__ void put_partials64(const Desc& d, int lb, int red, double (&v)[NC], Shared& sh) {
  static_assert(NC >= 1 && NC <= 3, "one to three components per reduction");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int E = (int)__reduce_max_sync(0xffffffffu, (unsigned)fx64_exponent(v[c]));
    const long long S = warp_sum57(E < fx::kBadExp ? fx64_image(v[c], E) : 0ll);
    if (lane == 0) {
      sh.whi[c][warp] = S;
      sh.wexp[c][warp] = E;
    }
  }
  if (threadIdx.x == 0) sh.tflag = 1;
  __syncthreads();
  for (int c = warp; c < NC; c += nw) {
    long long sw = 0;
    int ew = 1;
    if (lane < nw) {
      sw = sh.whi[c][lane];
      ew = sh.wexp[c][lane];
    }
    const int E = (int)__reduce_max_sync(0xffffffffu, (unsigned)ew);
    const long long y = E < fx::kBadExp ? (sw >> min(E - ew + 5, 63)) : 0ll;   // |y| < 2^57
    const long long S = warp_sum57(y);
    if (lane == 0) store_slot64(tag_slot(d, red, c, lb), S, E, red);
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
//
// SHIFT places the slot's mantissa: a slot holds m 2^(E + SHIFT - 1129)
// (the 64-bit block partials of put_partials64: kSlot64Shift).
template <int SHIFT>
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
  total = E < fx::kBadExp ? fx::to_double(t, E + SHIFT) : fx::to_double(0, fx::kBadExp);
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
  if (d.tagged) put_partials64<NC>(d, lb, red, v, sh);
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
    if (!tagged_total<kSlot64Shift>(d, red, c, t)) {
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

// Offset in a padded box of row length Ba of stencil entry k: (angle, ring)
// steps (0,0), (+1,0), (-1,0), (0,+1), (0,-1), (+1,+1), (-1,-1).
__device__ __forceinline__ int stencil_offset(int k, int Ba) {
  return (k == 3 || k == 5 ? Ba : (k == 4 || k == 6 ? -Ba : 0)) + (k == 1 || k == 5 ? 1 : (k == 2 || k == 6 ? -1 : 0));
}

// y = K v over the block's own rows in the O-grid tile form: row i sits at
// box position pos[i] and reads its seven neighbours at fixed offsets of the
// padded box (own values, gathered halo values, zeros on the ring outside the
// domain); no column indices.  One row per thread; op(i, s) as for spmv_ext.
template <typename Op>
__device__ __forceinline__ void spmv_box(const int* __restrict__ pos, const double* __restrict__ planes, int chunk,
                                         const double* box, int Ba, int nloc, Op op) {
  const int o1 = stencil_offset(1, Ba), o2 = stencil_offset(2, Ba), o3 = stencil_offset(3, Ba);
  const int o4 = stencil_offset(4, Ba), o5 = stencil_offset(5, Ba), o6 = stencil_offset(6, Ba);
  for (int i = threadIdx.x; i < nloc; i += blockDim.x) {
    const int q = pos[i];
    double s = planes[i] * box[q];
    s = fma(planes[chunk + i], box[q + o1], s);
    s = fma(planes[2 * chunk + i], box[q + o2], s);
    s = fma(planes[3 * chunk + i], box[q + o3], s);
    s = fma(planes[4 * chunk + i], box[q + o4], s);
    s = fma(planes[5 * chunk + i], box[q + o5], s);
    s = fma(planes[6 * chunk + i], box[q + o6], s);
    op(i, s);
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
  // RES stencil (O-grid tiles): the product's input is the block's padded box;
  // own rows and halo entries sit at their box positions, and the seven
  // coefficient planes replace the CSR slice
  const bool st = RES && d.stencil;
  const int* spos = nullptr;    // stencil: box position of each own row
  const int* hpos = nullptr;    // stencil: box position of each halo entry
  int Ba = 0;
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
    ext = base + 9 * chunk;                  // CSR: [chunk + halo_cap] own u, then gathered halo u; stencil: [box_cap]
    double* dh = ext + (st ? d.box_cap : chunk + d.halo_cap);   // [halo_cap]
    double* val = dh + d.halo_cap;           // CSR: [nnz_cap]; stencil: [7][chunk] planes
    stR = val + (st ? 7 * chunk : d.res_nnz_cap);   // [halo_cap] each
    stW = stR + d.halo_cap;
    stS = stW + d.halo_cap;
    int* row = reinterpret_cast<int*>(stS + d.halo_cap);
    int* col = row + chunk + 1;
    int* hd = st ? row + chunk : col + d.res_nnz_cap;
    const int h0 = d.hptr[lb];
    nh = d.hptr[lb + 1] - h0;
    if (st) {
      int* hp = hd + d.halo_cap;
      Ba = d.bdim[lb];
      for (int q = tid; q < d.box_cap; q += bd) ext[q] = 0.0;   // the ring outside the domain stays zero
      for (int k = 0; k < 7; ++k)
        for (int i = tid; i < nloc; i += bd) val[k * chunk + i] = d.planes[(size_t)k * n + r0 + i];
      for (int i = tid; i < nloc; i += bd) row[i] = d.bpos[r0 + i];
      for (int h = tid; h < nh; h += bd) hp[h] = d.hpos[h0 + h];
      spos = row;
      hpos = hp;
    } else {
      const int k0 = nloc > 0 ? d.rowptr[r0] : 0;
      const int nnzl = nloc > 0 ? d.rowptr[r1] - k0 : 0;
      for (int i = tid; i <= nloc; i += bd) row[i] = d.rowptr[r0 + i] - k0;
      for (int k = tid; k < nnzl; k += bd) {
        col[k] = d.lcol[k0 + k];
        val[k] = d.val[k0 + k];
      }
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

  // where own row i and halo entry h live in the product's input
  auto own_at = [&](int i) { return st ? spos[i] : i; };
  auto halo_at = [&](int h) { return st ? hpos[h] : nloc + h; };
  auto product = [&](auto op) {
    if (st) spmv_box(spos, L.val, chunk, ext, Ba, nloc, op);
    else spmv_ext<T>(L.row, L.col, L.val, ext, nloc, op);
  };

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
        for (int i = tid; i < nloc; i += bd) ext[own_at(i)] = x[i];
        for (int h = tid; h < nh; h += bd) ext[halo_at(h)] = __ldcg(d.x + hid[h]);
        __syncthreads();
        product(op);
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
        for (int i = tid; i < nloc; i += bd) ext[own_at(i)] = u[i];
        for (int h = tid; h < nh; h += bd) ext[halo_at(h)] = dih[h] * __ldcg(R0 + hid[h]);
        __syncthreads();
        product(op);
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
    // sc[3] = 1 / gamma_old, sc[6] = 1 / alpha_old and sc[7] = sc[3] sc[6] are prepared off the critical path
    int k = 0;
    auto derive = [&](Shared& S) {
      const double g = S.tot[0], dl = S.tot[1], rr = S.tot[2];
      // the tests look at the bits (integer pipe): this thread's chain of FP64
      // operations is the latency of every iteration on GB300's narrow FP64 pipe
      int st = -1;
      if (!finite_bits(g) || !finite_bits(dl) || !finite_bits(rr)) st = CGP_ERR_NONFINITE;
      else if (nonneg_le(rr, S.sc[4])) st = CGP_OK;   // (r,r) and (tol |b|)^2 are >= 0
      else if (its + k >= d.max_it) st = CGP_ERR_NOT_CONVERGED;
      double beta = 0.0, alpha;
      if (k == 0) {
        alpha = g / dl;
      } else {   // dl - beta gamma / alpha_old with beta = gamma / gamma_old; sc[7] = 1 / (gamma_old alpha_old)
        beta = g * S.sc[3];
        alpha = g / fma(-g * g, S.sc[7], dl);
      }
      if (st < 0 && !(positive_bits(g) && positive_bits(alpha) && finite_bits(alpha))) st = CGP_ERR_BREAKDOWN;
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
        sh.sc[7] = sh.sc[3] * sh.sc[6];
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
        if (RES) ext[own_at(i)] = ui;
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
                ext[halo_at(h)] = dih[h] * fma(-alpha, sj, hR[q]);
              }
            }
            for (; h < nh; h += hs) {
              const double sj = k == 0 ? stW[h] : fma(beta, stS[h], stW[h]);
              ext[halo_at(h)] = dih[h] * fma(-alpha, sj, stR[h]);
            }
          }
        } else {
          for (int h = tid; h < nh; h += bd) ext[halo_at(h)] = halo_u(hid[h], dih[h]);
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
        product(op);
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

// FP64 Jacobi-PCG in the pipelined form of Ghysels and Vanroose on O-grid
// tiles (tuning flag bits 4 and 5, rows resident, at least 256 threads per
// block): the product of an iteration is formed while the iteration's one
// grid-wide reduction completes, so the reduction's latency hides behind
// FP64 work instead of adding to it.
//
// With u = D^-1 r, w = K u, m = D^-1 w and n = K m, the recurrences
//   z = n + beta z,  s = w + beta s,  r -= alpha s,  u = D^-1 r,
//   w -= alpha z,    p = u + beta p,  x += alpha p
// keep s = K p and z = K D^-1 s, and (r,u), (w,u), (r,r) are the scalars of
// the single-reduction form.  Iteration k of a block:
//   (A) all warps: z, s, r, u, w of the own rows with alpha_k, beta_k;
//       w_(k+1) published; the partial sums of (r,u), (w,u), (r,r) stored
//       in the block's tagged slots; the block's flag released (it counts
//       the block's published w);
//   (B) warps 0-2 poll every block's slots of their component, and thread 0
//       derives alpha_(k+1), beta_(k+1); meanwhile the other warps put
//       m = D^-1 w of the own rows into the box, form n = K m on the rows
//       whose stencil stays inside the tile, update p_k and x_(k+1), wait
//       (acquire) for the flags of the blocks that own the tile's halo, load
//       their w, and form n on the tile's edge rows.
// The loop has no grid barrier: the tagged slots carry the totals and the
// flags the halo.  A block rewrites a copy of w (two, by parity) or a bank
// of slots only after it has seen every block's partial sums of the
// reduction in between, which every block stores after reading the older
// copy.  The recurrences drift from b - K x sooner than the single-reduction
// form's: convergence is confirmed on the true residual, and a loss of
// positive alpha after the first iteration restarts from the true residual
// (at most kMaxRestarts times in all).
//
// On GB300 the form is bound by the FP64 pipe: 19 FP64 operations per row
// against the single-reduction form's 15 fill about 4.4 us of the iteration
// at 512x256 on 152 blocks, and the neighbours' flags arrive about when the
// tile's inner product ends, so the iteration (6.7 us) gains little on the
// single-reduction form (6.9 us) and a restart near tol 1e-8 takes the rest.
// It is selected with cgp_set_tuning only (cgp_autotune leaves it out).
constexpr int kPlMinBlock = 256;   // three polling warps and at least five computing ones
constexpr int kPlMaxNbr = 64;      // blocks owning a tile's halo rows (itself across the periodic seam)
constexpr int kPlMaxBlocks = 2048; // blocks of a launch (the owners' bitmap)

// Barrier of nthreads threads (whole warps) on barrier id (not 0, which
// __syncthreads uses); the warp's lanes are reconverged first.
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  __syncwarp();
  asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int T>
__device__ void solve_fp64_pl(const Desc& d, int lb, Shared& sh) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int nbr[kPlMaxNbr];
  __shared__ unsigned owners[kPlMaxBlocks / 32];
  __shared__ int n_nbr, n_in, hflag;
  const int tid = threadIdx.x, bd = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int chunk = (d.n + d.nblk - 1) / d.nblk;
  const int r0 = min(d.n, lb * chunk), r1 = min(d.n, r0 + chunk), nloc = r1 - r0;
  const size_t n = d.n;
  int* const timeout = &d.res->timeout;
  Group grp{d.bar, timeout, (unsigned)d.nblk, 0u, d.spin_ns};
  int red = 0;
  // published (global): r of a pass's first product; w by parity of the publication count
  double* const R0 = d.pub64;
  double* const W0 = d.pub64 + 2 * n;
  double* const W1 = d.pub64 + 3 * n;
  // shared memory: own vectors, seven coefficient planes, the padded box, D^-1 of the halo;
  // box positions of the own rows, the rows in product order (inside the tile, then its
  // edge), box positions and global rows of the halo entries
  double* base = reinterpret_cast<double*>(dsm);
  double* x = base;
  double* r = base + chunk;
  double* uA = base + 2 * chunk;   // u_k and u_(k+1) alternate
  double* uB = base + 3 * chunk;
  double* w = base + 4 * chunk;
  double* p = base + 5 * chunk;
  double* s = base + 6 * chunk;
  double* z = base + 7 * chunk;
  double* nv = base + 8 * chunk;
  double* dil = base + 9 * chunk;
  double* bp = base + 10 * chunk;
  double* planes = base + 11 * chunk;
  double* box = planes + 7 * chunk;
  double* dih = box + d.box_cap;
  int* spos = reinterpret_cast<int*>(dih + d.halo_cap);
  int* ord = spos + chunk;
  int* hpos = ord + chunk;
  int* hid = hpos + d.halo_cap;
  const int h0 = d.hptr[lb], nh = d.hptr[lb + 1] - h0;
  const int Ba = d.bdim[lb];
  if (!d.tpart || !d.nflag || bd < kPlMinBlock || d.nblk > kPlMaxBlocks || nh > d.halo_cap) {
    finish(d, lb, CGP_ERR_INVALID_ARG, 0, 0, 0.0, 0.0, 0.0);
    return;
  }
  for (int q = tid; q < d.box_cap; q += bd) box[q] = 0.0;
  for (int k = 0; k < 7; ++k)
    for (int i = tid; i < nloc; i += bd) planes[k * chunk + i] = d.planes[(size_t)k * n + r0 + i];
  for (int i = tid; i < nloc; i += bd) {
    spos[i] = d.bpos[r0 + i];
    dil[i] = d.dinv[r0 + i];
  }
  for (int h = tid; h < nh; h += bd) {
    const int j = d.hidx[h0 + h];
    hpos[h] = d.hpos[h0 + h];
    hid[h] = j;
    dih[h] = d.dinv[j];
  }
  for (int q = tid; q < kPlMaxBlocks / 32; q += bd) owners[q] = 0u;
  // this block's slots and flag start empty; the first group barrier orders
  // that before any block reads them
  if (tid < 6) *tag_slot(d, tid / 3, tid % 3, lb) = make_ulonglong2(0ull, 0ull);
  if (tid == 0) d.nflag[lb] = 0u;
  __syncthreads();
  // rows whose seven box neighbours are all own rows (marked in the box), and
  // the blocks that own the halo rows
  for (int i = tid; i < nloc; i += bd) box[spos[i]] = 1.0;
  for (int h = tid; h < nh; h += bd) {
    const int o = hid[h] / chunk;
    atomicOr(&owners[o >> 5], 1u << (o & 31));
  }
  __syncthreads();
  const int o1 = stencil_offset(1, Ba), o2 = stencil_offset(2, Ba), o3 = stencil_offset(3, Ba);
  const int o4 = stencil_offset(4, Ba), o5 = stencil_offset(5, Ba), o6 = stencil_offset(6, Ba);
  if (warp == 0) {
    const unsigned below = (1u << lane) - 1u;
    int cnt = 0;
    for (int pass = 0; pass < 2; ++pass) {   // the tile's inner rows, then its edge rows, each in row order
      for (int b0 = 0; b0 < nloc; b0 += 32) {
        const int i = b0 + lane;
        bool take = false;
        if (i < nloc) {
          const int q = spos[i];
          const bool inner = box[q + o1] == 1.0 && box[q + o2] == 1.0 && box[q + o3] == 1.0 &&
                             box[q + o4] == 1.0 && box[q + o5] == 1.0 && box[q + o6] == 1.0;
          take = pass == 0 ? inner : !inner;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        if (take) ord[cnt + __popc(bal & below)] = i;
        cnt += __popc(bal);
      }
      if (pass == 0 && lane == 0) n_in = cnt;
    }
  } else if (warp == 1 && lane == 0) {
    int c = 0;
    for (int q = 0; q < (d.nblk + 31) / 32; ++q)
      for (unsigned bits = owners[q]; bits; bits &= bits - 1u) {
        if (c < kPlMaxNbr) nbr[c] = 32 * q + __ffs(bits) - 1;
        ++c;
      }
    n_nbr = c;
  }
  __syncthreads();
  if (n_nbr > kPlMaxNbr) {
    finish(d, lb, CGP_ERR_INVALID_ARG, 0, 0, 0.0, 0.0, 0.0);
    return;
  }
  for (int q = tid; q < d.box_cap; q += bd) box[q] = 0.0;   // the ring outside the domain stays zero
  const int ni = n_in;

  // the product's row i from the box (own values, halo values, zeros on the ring)
  auto stencil_at = [&](int i) {
    const int q = spos[i];
    double a = planes[i] * box[q];
    a = fma(planes[chunk + i], box[q + o1], a);
    a = fma(planes[2 * chunk + i], box[q + o2], a);
    a = fma(planes[3 * chunk + i], box[q + o3], a);
    a = fma(planes[4 * chunk + i], box[q + o4], a);
    a = fma(planes[5 * chunk + i], box[q + o5], a);
    return fma(planes[6 * chunk + i], box[q + o6], a);
  };

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
      d.x[r0 + i] = xi;
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
  if (tid == 0) sh.sc[4] = stop2;

  int its = 0, restarts = 0, status = CGP_ERR_NOT_CONVERGED, pending = -1;
  unsigned pub = 0;   // publications of w so far (the same count in every block)
  double rr_rec = 0.0, rr_true = 0.0;
  bool first = true;

  // scalars of reduction kk (thread 0): sc[0] alpha, sc[1] beta, sc[2] gamma, sc[5] (r,r), isc[0]
  // stop flag; sc[3] = 1 / gamma_old, sc[7] = 1 / (gamma_old alpha_old) come from thread 32
  auto derive = [&](int kk) {
    const double g = sh.tot[0], dl = sh.tot[1], rr = sh.tot[2];
    int st = -1;
    if (!finite_bits(g) || !finite_bits(dl) || !finite_bits(rr)) st = CGP_ERR_NONFINITE;
    else if (nonneg_le(rr, sh.sc[4])) st = CGP_OK;
    else if (its + kk >= d.max_it) st = CGP_ERR_NOT_CONVERGED;
    double beta = 0.0, alpha;
    if (kk == 0) {
      alpha = g / dl;
    } else {
      beta = g * sh.sc[3];
      alpha = g / fma(-g * g, sh.sc[7], dl);
    }
    if (st < 0 && !(positive_bits(g) && positive_bits(alpha) && finite_bits(alpha))) st = CGP_ERR_BREAKDOWN;
    sh.isc[0] = st;
    sh.sc[0] = alpha;
    sh.sc[1] = beta;
    sh.sc[2] = g;
    sh.sc[5] = rr;
  };
  // (B) of reduction kk, whose partials the block has stored and whose w is the pub-th
  // publication: warps 0-2 poll the slots, thread 0 derives; the other warps form n = K D^-1 w
  // and, when px, p_(kk-1) and x_kk from u_(kk-1) (uc) with the previous scalars
  auto phase_b = [&](int kk, bool px, double alpha, double beta, const double* uc) -> bool {
    if (warp < 3) {
      if (tid == 32 && kk > 0) {
        sh.sc[3] = 1.0 / sh.sc[2];
        sh.sc[6] = 1.0 / sh.sc[0];
        sh.sc[7] = sh.sc[3] * sh.sc[6];
      }
      double t;
      if (!tagged_total<kSlot64Shift>(d, red, warp, t)) {
        if (lane == 0) sh.tflag = 0;
      } else if (lane == 0) {
        sh.tot[warp] = t;
      }
      named_sync(2, 96);
      if (tid == 0 && sh.tflag) derive(kk);
    } else {
      const int t0 = tid - 96, nt = bd - 96;
      const double* Wp = (pub & 1) ? W1 : W0;
      for (int i = t0; i < nloc; i += nt) box[spos[i]] = dil[i] * w[i];
      named_sync(1, nt);
      for (int j = t0; j < ni; j += nt) {
        const int i = ord[j];
        nv[i] = stencil_at(i);
      }
      if (px) {
        for (int i = t0; i < nloc; i += nt) {
          const double pi = kk == 1 ? uc[i] : fma(beta, p[i], uc[i]);
          p[i] = pi;
          x[i] = fma(alpha, pi, x[i]);
        }
      }
      if (t0 < n_nbr && !wait_at_least(d.nflag + nbr[t0], pub, timeout, d.spin_ns)) hflag = 0;
      named_sync(1, nt);
      if (hflag) {
        for (int h = t0; h < nh; h += nt) box[hpos[h]] = dih[h] * __ldcg(Wp + hid[h]);
        named_sync(1, nt);
        for (int j = ni + t0; j < nloc; j += nt) {
          const int i = ord[j];
          nv[i] = stencil_at(i);
        }
      }
    }
    __syncthreads();
    return sh.tflag && hflag;
  };

  while (true) {
    // ---- true residual of the published x: r = bp - K x, u = D^-1 r; r published ----
    {
      double v1[1] = {0.0};
      for (int i = tid; i < nloc; i += bd) box[spos[i]] = x[i];
      for (int h = tid; h < nh; h += bd) box[hpos[h]] = __ldcg(d.x + hid[h]);
      __syncthreads();
      for (int i = tid; i < nloc; i += bd) {
        const double t = bp[i] - stencil_at(i);
        r[i] = t;
        uA[i] = dil[i] * t;
        R0[r0 + i] = t;
        v1[0] += t * t;
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

    // ---- w_0 = K u_0 (halo u_j = D^-1_j r_j), published; the first reduction and n_0 ----
    {
      ++pub;
      double* Wp = (pub & 1) ? W1 : W0;
      double v3[3] = {0.0, 0.0, 0.0};
      for (int i = tid; i < nloc; i += bd) box[spos[i]] = uA[i];
      for (int h = tid; h < nh; h += bd) box[hpos[h]] = dih[h] * __ldcg(R0 + hid[h]);
      __syncthreads();
      for (int i = tid; i < nloc; i += bd) {
        const double a = stencil_at(i);
        w[i] = a;
        Wp[r0 + i] = a;
        const double ui = uA[i], ri = r[i];
        v3[0] += ri * ui;
        v3[1] += a * ui;
        v3[2] += ri * ri;
      }
      if (tid == 0) hflag = 1;
      put_partials64<3>(d, lb, red, v3, sh);   // its block barrier also orders the box reads above
      if (tid == 0) st_release_u32(d.nflag + lb, pub);
    }
    if (!phase_b(0, false, 0.0, 0.0, nullptr)) return;
    ++red;
    int k = 0;
    double* uc = uA;   // u_k
    double* un = uB;   // u_(k+1)
    while (true) {
      const int st = sh.isc[0];
      if (st >= 0) {
        if (st == CGP_ERR_BREAKDOWN && k > 0) break;   // the recurrences drifted: restart from the true residual
        if (st != CGP_OK) pending = st;
        break;
      }
      // (A) z_k, s_k, r_(k+1), u_(k+1), w_(k+1) of the own rows; w published; partials; flag
      const double alpha = sh.sc[0], beta = sh.sc[1];
      ++pub;
      double* Wp = (pub & 1) ? W1 : W0;
      double v3[3] = {0.0, 0.0, 0.0};
      for (int i = tid; i < nloc; i += bd) {
        const double zi = k == 0 ? nv[i] : fma(beta, z[i], nv[i]);
        const double si = k == 0 ? w[i] : fma(beta, s[i], w[i]);
        z[i] = zi;
        s[i] = si;
        const double ri = fma(-alpha, si, r[i]);
        r[i] = ri;
        const double ui = dil[i] * ri;
        un[i] = ui;
        const double wi = fma(-alpha, zi, w[i]);
        w[i] = wi;
        Wp[r0 + i] = wi;
        v3[0] += ri * ui;
        v3[1] += wi * ui;
        v3[2] += ri * ri;
      }
      if (tid == 0) hflag = 1;
      put_partials64<3>(d, lb, red, v3, sh);
      if (tid == 0) st_release_u32(d.nflag + lb, pub);
      // (B) n_(k+1), p_k and x_(k+1) while the reduction of iteration k + 1 completes
      if (!phase_b(k + 1, true, alpha, beta, uc)) return;
      ++red;
      ++k;
      double* t = uc;
      uc = un;
      un = t;
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
      d.x[r0 + i] = xi;
    }
    if (!grp.sync(sh)) return;
  }
  finish(d, lb, status, its, restarts, sqrt(rr_rec) / bnorm, sqrt(rr_true) / bnorm, bnorm);
}

// ---------------------------------------------------------------------------
// FP32 reductions of the inner solve: warp trees on the FP32 pipe, one slot
// per block, every block sums the slots in the same order (deterministic).
// ---------------------------------------------------------------------------
// Tagged FP32 partials (tuning flag bit 3): the partial of component c of
// reduction red from block blk is one 64-bit word, the FP32 bits low and
// red + 1 high, in the tagged-slot area (a single-copy atomic store; the
// block zeroes its words at launch start).  Banks by the reduction's parity.
__device__ __forceinline__ unsigned long long* ftag_slot(const Desc& d, int red, int c, int blk) {
  return reinterpret_cast<unsigned long long*>(d.tpart) + ((size_t)((red & 1) * 3 + c) * d.part_stride + blk);
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

template <int NC>
__device__ __forceinline__ void put_partials_f(const Desc& d, int lb, int red, const float (&v)[NC], Shared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const float s = warp_sum(v[c]);
    if (lane == 0) sh.fred[c][warp] = s;
  }
  if (d.tagged && threadIdx.x == 0) sh.tflag = 1;
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float s = lane < nw ? sh.fred[c][lane] : 0.0f;
      s = warp_sum(s);
      if (lane == 0) {
        if (d.tagged)
          st_relaxed_u64(ftag_slot(d, red, c, lb),
                         ((unsigned long long)(unsigned)(red + 1) << 32) | (unsigned long long)__float_as_uint(s));
        else
          d.fpart[((red & 1) * NCOMP + c) * d.part_stride + lb] = s;
      }
    }
  }
}

// One warp: component c of tagged FP32 reduction red, summed in the order
// of get_totals_f_then (lane l adds blocks l, l + 32, ..., then a butterfly):
// the same bits.  Each lane polls its words with relaxed loads, all issued
// before any is examined, until they carry the tag.  Gives up (false on every
// lane) after d.spin_ns or when another block has given up.
__device__ __forceinline__ bool ftagged_total(const Desc& d, int red, int c, float& total) {
  constexpr int PRE = 8;
  const int lane = threadIdx.x & 31;
  const unsigned tag = (unsigned)(red + 1);
  int* const timeout = &d.res->timeout;
  float acc = 0.0f;
  unsigned long long t0 = 0;
  unsigned spins = 0;
  for (int base = 0; base < d.nblk; base += 32 * PRE) {
    unsigned long long w[PRE];
    unsigned pend = 0;
#pragma unroll
    for (int t = 0; t < PRE; ++t) {
      w[t] = 0ull;
      if (base + lane + 32 * t < d.nblk) pend |= 1u << t;
    }
    const unsigned have = pend;
    while (true) {
      const unsigned pm = pend;
#pragma unroll
      for (int t = 0; t < PRE; ++t)
        if (pm & (1u << t)) w[t] = ld_relaxed_u64(ftag_slot(d, red, c, base + lane + 32 * t));
#pragma unroll
      for (int t = 0; t < PRE; ++t)
        if ((pm & (1u << t)) && (unsigned)(w[t] >> 32) == tag) pend &= ~(1u << t);
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
#pragma unroll
    for (int t = 0; t < PRE; ++t)
      if (have & (1u << t)) acc += __uint_as_float((unsigned)w[t]);
  }
  total = warp_sum(acc);
  return true;
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

// Finish of an FP32 inner reduction, after put_partials_f and grp.arrive().
// Untagged: the barrier, then warp 0 reads the slots (get_totals_f_then)
// while the other threads run stage().  Tagged (d.tagged): warps 0 .. NC-1
// poll the tagged words while one more thread waits on the barrier, so the
// totals are known when it completes; then stage() and the derivation.
template <int NC, typename F, typename G>
__device__ __forceinline__ bool red_finish_f(const Desc& d, Group& grp, int red, Shared& sh, F derive, G stage) {
  if (!d.tagged) {
    if (!grp.wait(sh)) return false;
    stage();
    get_totals_f_then<NC>(d, red, sh, derive);
    return true;
  }
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < NC; c += nw) {
    float t;
    if (!ftagged_total(d, red, c, t)) {
      if ((threadIdx.x & 31) == 0) sh.tflag = 0;
      break;
    }
    if ((threadIdx.x & 31) == 0) sh.ftot[c] = t;
  }
  if (threadIdx.x == (nw > NC ? 32 * NC : 0) && !grp.wait_one()) sh.tflag = 0;
  __syncthreads();
  if (!sh.tflag) return false;
  stage();
  if (threadIdx.x == 0) derive(sh);
  __syncthreads();
  return true;
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

  // tagged inner reductions: this block's words start empty; the first
  // barrier orders that before any block reads them
  if (d.tagged && tid < 6) *ftag_slot(d, tid / 3, tid % 3, lb) = 0ull;
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
      grp.arrive();   // finished below by red_finish_f (nothing in between writes what other blocks read)
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
    // RES: after the barrier, the threads above the reduction's warps stage
    // the halo inputs r_j, w_j, s_j of the coming iteration.  Untagged, into
    // shared memory while warp 0 fetches the totals (the two global round
    // trips overlap).  Tagged, the totals are already known: a thread's first
    // HREG entries go to registers and are consumed by the same thread after
    // the own-row update, so the loads overlap the derivation and that update;
    // further entries go through shared memory (the same thread reads them).
    constexpr int HREG = 2;
    const int TWs = d.tagged ? 96 : 32;
    const bool staged = RES && bd > TWs;
    float hR[HREG], hW[HREG], hS[HREG];
#pragma unroll
    for (int q = 0; q < HREG; ++q) hR[q] = hW[q] = hS[q] = 0.0f;
    auto stage = [&](int kk) {
      if (!staged || tid < TWs) return;
      const float* Rc = (kk & 1) ? R1 : R0;
      const float* Wc = (kk & 1) ? W1 : W0;
      const float* Sc = (kk & 1) ? S1 : S0;
      const int hs = bd - TWs;
      int h = tid - TWs;
      if (d.tagged) {
#pragma unroll
        for (int q = 0; q < HREG; ++q, h += hs) {
          if (h < nh) {
            const int j = hid[h];
            hR[q] = __ldcg(Rc + j);
            hW[q] = __ldcg(Wc + j);
            if (kk > 0) hS[q] = __ldcg(Sc + j);
          }
        }
      }
      for (; h < nh; h += hs) {
        const int j = hid[h];
        stR[h] = __ldcg(Rc + j);
        stW[h] = __ldcg(Wc + j);
        if (kk > 0) stS[h] = __ldcg(Sc + j);
      }
    };
    if (!red_finish_f<3>(d, grp, red, sh, derive, [&] { stage(0); })) return;
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
      // own rows: s, r and u_(k+1) (RES: into the product's input, while iu
      // keeps u_k for the update of p and e during the reduction's wait; without
      // RES also p and e here)
      for (int i = tid; i < nloc; i += bd) {
        const float si = k == 0 ? iw[i] : fmaf(beta, is[i], iw[i]);
        if (!RES) {
          const float pi = k == 0 ? iu[i] : fmaf(beta, ip[i], iu[i]);
          ip[i] = pi;
          ie[i] = fmaf(alpha, pi, ie[i]);
        }
        is[i] = si;
        const float ri = fmaf(-alpha, si, ir[i]);
        ir[i] = ri;
        if (RES) ext[i] = di[i] * ri;
        else iu[i] = di[i] * ri;
        Rn[r0 + i] = ri;
        Sn[r0 + i] = si;
      }
      // halo: u_j = D^-1_j (r_j - alpha (w_j + beta s_j)) from the owner's published values
      auto halo_u = [&](int j, float dj) {
        const float sj = k == 0 ? __ldcg(Wc + j) : fmaf(beta, __ldcg(Sc + j), __ldcg(Wc + j));
        return dj * fmaf(-alpha, sj, __ldcg(Rc + j));
      };
      if constexpr (RES) {
        if (staged && d.tagged) {
          if (tid >= TWs) {   // the entries this thread staged
            const int hs = bd - TWs;
            int h = tid - TWs;
#pragma unroll
            for (int q = 0; q < HREG; ++q, h += hs) {
              if (h < nh) {
                const float sj = k == 0 ? hW[q] : fmaf(beta, hS[q], hW[q]);
                ext[nloc + h] = dih[h] * fmaf(-alpha, sj, hR[q]);
              }
            }
            for (; h < nh; h += hs) {
              const float sj = k == 0 ? stW[h] : fmaf(beta, stS[h], stW[h]);
              ext[nloc + h] = dih[h] * fmaf(-alpha, sj, stR[h]);
            }
          }
        } else if (staged) {
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
        const float u = RES ? ext[il] : iu[il], r = ir[il];
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
      grp.arrive();
      if constexpr (RES) {   // p_k = u_k + beta p_(k-1), e += alpha p_k, then u_(k+1), while the other blocks arrive
        for (int i = tid; i < nloc; i += bd) {
          const float pi = k == 0 ? iu[i] : fmaf(beta, ip[i], iu[i]);
          ip[i] = pi;
          ie[i] = fmaf(alpha, pi, ie[i]);
          iu[i] = ext[i];
        }
      }
      ++k;
      if (!red_finish_f<3>(d, grp, red, sh, derive, [&] { stage(k); })) return;
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

}  // namespace
}  // namespace cgp
