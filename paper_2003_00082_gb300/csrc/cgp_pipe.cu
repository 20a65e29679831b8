// Pipelined FP64 Jacobi-PCG (tuning flag bit 4): the single-system and
// batched kernels of the solve loop in which each iteration's grid-wide
// reduction completes while the next product is formed.  Rows resident in
// shared memory only; lanes per row 1, 2 or 4.
#include "cgp_solver.cuh"

namespace cgp {
namespace {

// ---- shared-memory mbarriers (arrive with release, bounded waits with acquire) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(unsigned long long* mb, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}

__device__ __forceinline__ void mb_arrive(unsigned long long* mb) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(mb)) : "memory");
}

__device__ __forceinline__ void mb_inval(unsigned long long* mb) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(mb)) : "memory");
}

__device__ __forceinline__ bool mb_test(unsigned long long* mb, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(mb)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait (one thread) until the phase of parity `parity` of mbarrier mb has
// completed.  Gives up after spin_ns of wall-clock time, or as soon as
// another block has given up (the solve's timeout word): false then.
__device__ __forceinline__ bool mb_wait(unsigned long long* mb, unsigned parity, int* timeout, long long spin_ns) {
  unsigned long long t0 = 0;
  unsigned spins = 0;
  while (!mb_test(mb, parity)) {
    if ((++spins & 255u) == 0) {
      if (*(volatile int*)timeout) return false;
      const unsigned long long now = global_ns();
      if (t0 == 0) {
        t0 = now;
      } else if ((long long)(now - t0) > spin_ns) {
        atomicExch(timeout, 1);
        return false;
      }
    }
  }
  return true;
}

// The same wait for a whole warp: lane 0 waits, the warp synchronises (so
// every lane's later reads follow lane 0's acquire), the result on every lane.
__device__ __forceinline__ bool mb_wait_warp(unsigned long long* mb, unsigned parity, int* timeout, long long spin_ns) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mb_wait(mb, parity, timeout, spin_ns);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  __syncwarp();
  return ok;
}

// ---- published vectors as tagged words ----
// A published value goes out as one 128-bit store whose two 64-bit halves
// each carry 32 bits of the value and the same 32-bit tag (the restart pass
// and the iteration).  Each half is single-copy atomic, so a reader that
// finds the expected tag in both halves holds the value of that store; a
// reader polls until it does.  No grid barrier or release fence is needed.
__device__ __forceinline__ unsigned pipe_tag(int pass, int k) { return ((unsigned)pass << 24) | (unsigned)(k + 1); }

__device__ __forceinline__ void publish(ulonglong2* slot, double v, unsigned tag) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  st_relaxed_b128(slot, ((unsigned long long)tag << 32) | (b & 0xFFFFFFFFull), ((unsigned long long)tag << 32) | (b >> 32));
}

__device__ __forceinline__ bool tag_ok(const ulonglong2& w, unsigned tag) {
  return (unsigned)(w.x >> 32) == tag && (unsigned)(w.y >> 32) == tag;
}

__device__ __forceinline__ double tagged_value(const ulonglong2& w) {
  return __longlong_as_double((long long)((w.y << 32) | (w.x & 0xFFFFFFFFull)));
}

// Block-private state of the pipelined loop (besides the dynamic rows).
// Each mbarrier completes one phase per iteration, so a waiter of iteration k
// waits for parity k & 1; no phase can complete twice before its waiters have
// seen it (every arrival for iteration k + 1 follows a wait on iteration k's
// outcome, or on the consumer's arrival, as noted at each use).
struct PipeShared {
  unsigned long long mb_part;    // compute warps' partial sums written (one arrival per compute warp)
  unsigned long long mb_ext;     // the product's input complete, the staged halo consumed (per compute warp)
  unsigned long long mb_end;     // compute warps past the product and the p, x update (per compute warp)
  unsigned long long mb_stage;   // halo inputs staged (the staging warp)
  unsigned long long mb_tot;     // the three components' totals written (the reduction warps)
  unsigned long long mb_scal;    // the iteration's scalars known (reduction warp 0)
  long long ws[3][32];           // per compute warp: fixed-point partial of each component
  int we[3][32];
  double tot[3];                 // totals of the iteration's reduction
  double alpha, beta;            // scalars of the iteration
  int status;                    // -1 continue, else a status (or kRestartCode)
  int iter_done;                 // last iteration whose scalars are known (-1 before the first)
  int fail;                      // a wait gave up
};

// FP64 Jacobi-PCG in the pipelined form of Ghysels and Vanroose (tuning flag
// bit 4, rows resident in shared memory, at least 256 threads per block):
// the iteration's one grid-wide reduction completes while the next product
// is formed.
//
// With u = D^-1 r, w = K u, m = D^-1 w and n = K m, the recurrences
//   z = n + beta z,  s = w + beta s,  p = u + beta p,
//   x += alpha p,  r -= alpha s,  u = D^-1 r,  w -= alpha z
// keep s = K p and z = K D^-1 s, so (r,u), (w,u) and (r,r) of iteration k
// (the same scalars as the single-reduction form) can be reduced while
// n_k = K D^-1 w_k is computed.
//
// The warps of a block split the work of iteration k:
//   compute warps (4 ..): z, s, r, u, w with the previous scalars (w_k and
//     z_(k-1) published); partial (r,u), (w,u), (r,r) per warp; m = D^-1 w
//     on the own rows and on the staged halo (w_j rebuilt from the owner's
//     published w, n, z with the owner's own operations, so the bits agree);
//     n_k = K m (published); p_(k-1) and x_k; then the new scalars
//   reduction warps (0 - 2, one component each): fold the compute warps'
//     partials, store the block's tagged slot, poll every block's slot of
//     the reduction and sum; warp 0 derives alpha_k, beta_k and the stop test
//   staging warp (3): poll the halo rows' published words of the coming
//     iteration until their tags are current and copy the values to shared
//     memory
// so the reduction's round trip and the halo exchange overlap the compute
// warps' FP64 work.  The roles meet on shared-memory mbarriers; every wait
// has a time limit.
//
// Published words: W, Z and N in three copies each, by iteration.  A copy
// is rewritten three iterations later; by then every block has staged it
// (rewriting iteration k's copy needs the scalars of iteration k + 2, hence
// every block's partial sums of k + 2, which its compute warps form only
// after consuming their staged halo of k + 1, staged after that of k).  As
// in the single-reduction form, convergence of the recursive residual is
// confirmed on the true residual, with a restart from it otherwise; a loss
// of positive alpha after the first iteration (the recurrences drifted by
// rounding) also restarts from the true residual.
constexpr int kRestartCode = 1000;   // not a status: leave the iteration and restart from the true residual
constexpr int kPipeRoleWarps = 4;    // reduction warps 0..2 and the staging warp 3

template <int T>
__device__ void solve_fp64_pipe(const Desc& d, int lb, Shared& sh) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ PipeShared ps;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int chunk = (d.n + d.nblk - 1) / d.nblk;
  const int r0 = min(d.n, lb * chunk), r1 = min(d.n, r0 + chunk), nloc = r1 - r0;
  const size_t n = d.n;
  int* const timeout = &d.res->timeout;
  Group grp{d.bar, timeout, (unsigned)d.nblk, 0u, d.spin_ns};
  int red = 0;

  // published words: W[3], Z[3], N[3], each [n] 128-bit
  ulonglong2* const Wt = reinterpret_cast<ulonglong2*>(d.pub64);
  ulonglong2* const Zt = Wt + 3 * n;
  ulonglong2* const Nt = Wt + 6 * n;
  double* const U0 = d.z;               // u_0 of a pass, published for the first product

  // shared memory: own vectors, the product's input [own | halo], halo D^-1,
  // staged halo inputs, CSR slice
  double* base = reinterpret_cast<double*>(dsm);
  double* x = base;
  double* r = base + chunk;
  double* uA = base + 2 * chunk;         // u_k and u_(k+1) alternate
  double* uB = base + 3 * chunk;
  double* w = base + 4 * chunk;
  double* p = base + 5 * chunk;
  double* sv = base + 6 * chunk;
  double* z = base + 7 * chunk;
  double* nv = base + 8 * chunk;
  double* dil = base + 9 * chunk;
  double* bp = base + 10 * chunk;
  double* ext = base + 11 * chunk;       // [chunk + halo_cap]
  double* dih = ext + chunk + d.halo_cap;
  double* stW = dih + d.halo_cap;        // staged halo w, n, z of the coming iteration
  double* stN = stW + d.halo_cap;
  double* stZ = stN + d.halo_cap;
  double* val = stZ + d.halo_cap;
  int* row = reinterpret_cast<int*>(val + d.res_nnz_cap);
  int* col = row + chunk + 1;
  int* hid = col + d.res_nnz_cap;
  const int k0 = nloc > 0 ? d.rowptr[r0] : 0;
  const int nnzl = nloc > 0 ? d.rowptr[r1] - k0 : 0;
  const int h0 = d.hptr[lb];
  const int nh = d.hptr[lb + 1] - h0;
  for (int i = tid; i <= nloc; i += bd) row[i] = d.rowptr[r0 + i] - k0;
  for (int k = tid; k < nnzl; k += bd) {
    col[k] = d.lcol[k0 + k];
    val[k] = d.val[k0 + k];
  }
  for (int h = tid; h < nh; h += bd) {
    const int j = d.hidx[h0 + h];
    hid[h] = j;
    dih[h] = d.dinv[j];
  }
  for (int i = tid; i < nloc; i += bd) dil[i] = d.dinv[r0 + i];
  if (!d.tpart || bd < 32 * (kPipeRoleWarps + 4) || d.max_it >= (1 << 24)) {
    finish(d, lb, CGP_ERR_INVALID_ARG, 0, 0, 0.0, 0.0, 0.0);
    return;
  }
  if (tid < 6) *tag_slot(d, tid / 3, tid % 3, lb) = make_ulonglong2(0ull, 0ull);
  // this block's published words start untagged (the first grid barrier orders
  // that before any block polls them)
  for (int q = 0; q < 9; ++q)
    for (int i = tid; i < nloc; i += bd) Wt[(size_t)q * n + r0 + i] = make_ulonglong2(0ull, 0ull);

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

  // roles of the pipelined loop
  const int ctid = tid - 32 * kPipeRoleWarps;     // compute threads: ctid >= 0
  const int nct = bd - 32 * kPipeRoleWarps;
  const int ncw = nct >> 5;

  int its = 0, restarts = 0, status = CGP_ERR_NOT_CONVERGED, pending = -1, pass = 0;
  double rr_rec = 0.0, rr_true = 0.0;
  bool first = true;
  while (true) {
    // ---- true residual of the projected, published x: r = bp - K x, u_0 = D^-1 r (published) ----
    {
      double v1[1] = {0.0};
      for (int i = tid; i < nloc; i += bd) ext[i] = x[i];
      for (int h = tid; h < nh; h += bd) ext[nloc + h] = __ldcg(d.x + hid[h]);
      __syncthreads();
      spmv_ext<T>(row, col, val, ext, nloc, [&](int il, double sum) {
        const double t = bp[il] - sum;
        r[il] = t;
        const double ui = dil[il] * t;
        uA[il] = ui;
        U0[r0 + il] = ui;
        v1[0] += t * t;
      });
      red_start<1>(d, grp, lb, red, v1, sh);
      if (!red_finish<1>(d, grp, red, sh)) return;
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
    ++pass;

    // ---- w_0 = K u_0 (halo u from the published u_0), published as tagged W[0] ----
    for (int i = tid; i < nloc; i += bd) ext[i] = uA[i];
    for (int h = tid; h < nh; h += bd) ext[nloc + h] = __ldcg(U0 + hid[h]);
    if (tid == 0) {
      mb_init(&ps.mb_part, (unsigned)ncw);
      mb_init(&ps.mb_ext, (unsigned)ncw);
      mb_init(&ps.mb_end, (unsigned)ncw);
      mb_init(&ps.mb_stage, 1u);
      mb_init(&ps.mb_tot, 3u);
      mb_init(&ps.mb_scal, 1u);
      ps.fail = 0;
      ps.status = -1;
      ps.iter_done = -1;
    }
    __syncthreads();
    spmv_ext<T>(row, col, val, ext, nloc, [&](int il, double sum) {
      w[il] = sum;
      publish(Wt + r0 + il, sum, pipe_tag(pass, 0));
    });
    __syncthreads();

    const int red0 = red;   // reduction k of the loop is red0 + k
    int k = 0;
    if (warp < 3) {
      // ================= reduction warps: component `warp` of every iteration's reduction =================
      double g_inv = 0.0, a_inv = 0.0;   // warp 0, lane 0: 1 / gamma and 1 / alpha of the previous iteration
      while (true) {
        // the compute warps' partials of reduction k
        if (!mb_wait_warp(&ps.mb_part, (unsigned)(k & 1), timeout, d.spin_ns) && lane == 0) ps.fail = 1;
        {
          long long sw = 0;
          int ew = 1;
          if (lane < ncw) {
            sw = ps.ws[warp][lane];
            ew = ps.we[warp][lane];
          }
          const int E = (int)__reduce_max_sync(0xffffffffu, (unsigned)ew);
          const long long y = E < fx::kBadExp ? (sw >> min(E - ew + 5, 63)) : 0ll;   // |y| < 2^57
          const long long S = warp_sum57(y);
          if (lane == 0) store_slot64(tag_slot(d, red, warp, lb), S, E, red);
        }
        double t = 0.0;
        const bool ok = tagged_total<kSlot64Shift>(d, red, warp, t);
        if (lane == 0) {
          ps.tot[warp] = t;
          if (!ok) ps.fail = 1;
          mb_arrive(&ps.mb_tot);   // warps 1 and 2 arrive for iteration k + 1 only after seeing scal(k)
        }
        // warp 0: the three totals; warps 1 and 2: the outcome warp 0 derives from them
        if (!mb_wait_warp(warp == 0 ? &ps.mb_tot : &ps.mb_scal, (unsigned)(k & 1), timeout, d.spin_ns) && lane == 0)
          ps.fail = 1;
        if (warp == 0 && lane == 0) {   // the scalars, then 1 / gamma and 1 / alpha for the next beta
          const double g = ps.tot[0], dl = ps.tot[1], rr = ps.tot[2];
          int st = -1;
          if (ps.fail) st = CGP_ERR_TIMEOUT;
          else if (!isfinite(g) || !isfinite(dl) || !isfinite(rr)) st = CGP_ERR_NONFINITE;
          else if (rr <= stop2) st = CGP_OK;
          else if (its + k >= d.max_it) st = CGP_ERR_NOT_CONVERGED;
          double beta = 0.0, alpha;
          if (k == 0) {
            alpha = g / dl;
          } else {
            beta = g * g_inv;
            alpha = g / (dl - beta * g * a_inv);
          }
          // after the first iteration a non-positive alpha means the recurrences drifted from K u
          if (st < 0 && !(g > 0.0 && alpha > 0.0 && isfinite(alpha))) st = k > 0 ? kRestartCode : CGP_ERR_BREAKDOWN;
          if (ps.fail) st = CGP_ERR_TIMEOUT;
          ps.alpha = alpha;
          ps.beta = beta;
          ps.status = st;
          __threadfence_block();
          *(volatile int*)&ps.iter_done = k;
          mb_arrive(&ps.mb_scal);
          g_inv = 1.0 / g;
          a_inv = 1.0 / alpha;
        }
        __syncwarp();
        const int st = *(volatile int*)&ps.status;
        ++red;
        ++k;
        if (st >= 0) break;
      }
    } else if (warp == 3) {
      // ================= staging warp: halo inputs of iteration j from the owners' published words =================
      for (int j = 0;; ++j) {
        if (j >= 2) {
          // iteration j - 1 (whose words iteration j needs) runs only if iteration j - 2 continued
          bool known = true;
          if (lane == 0) {
            unsigned long long t0 = 0;
            unsigned spins = 0;
            while (*(volatile int*)&ps.iter_done < j - 2) {
              if ((++spins & 255u) == 0) {
                if (*(volatile int*)timeout || *(volatile int*)&ps.fail) { known = false; break; }
                const unsigned long long now = global_ns();
                if (t0 == 0) t0 = now;
                else if ((long long)(now - t0) > d.spin_ns) { atomicExch(timeout, 1); known = false; break; }
              }
            }
          }
          known = __shfl_sync(0xffffffffu, known ? 1 : 0, 0) != 0;
          __syncwarp();
          if (!known) break;
          const int done = *(volatile int*)&ps.iter_done;
          if (done == j - 2 && *(volatile int*)&ps.status >= 0) break;   // the loop ended at iteration j - 2
        }
        // the compute warps have consumed the staging of iteration j - 1 (iteration j - 1 runs:
        // j - 1 is 0, or iteration j - 2 continued); they consume staging j only after this arrival
        if (j >= 1 && !mb_wait_warp(&ps.mb_ext, (unsigned)((j - 1) & 1), timeout, d.spin_ns)) {
          if (lane == 0) ps.fail = 1;
          break;
        }
        // w_(j-1), n_(j-1), z_(j-2) of every halo row (iteration 0: w_0)
        const int jw = j == 0 ? 0 : j - 1;
        const ulonglong2* Wp = Wt + (size_t)(jw % 3) * n;
        const ulonglong2* Np = Nt + (size_t)((j + 2) % 3) * n;
        const ulonglong2* Zp = Zt + (size_t)((j + 1) % 3) * n;
        const unsigned tw = pipe_tag(pass, jw), tz = pipe_tag(pass, j - 2);
        // up to kStageChunks x 32 halo rows per pass, every load of a pass in flight at once; each
        // round re-reads only the words whose tag is not yet current
        constexpr int kStageChunks = 3;
        bool ok = true;
        unsigned long long t0 = 0;
        unsigned spins = 0;
        for (int hb = 0; hb < nh && ok; hb += 32 * kStageChunks) {
          ulonglong2 a[kStageChunks], b[kStageChunks], c[kStageChunks];
          unsigned need = 0;   // bits: 3 q + {0: w, 1: n, 2: z}
#pragma unroll
          for (int q = 0; q < kStageChunks; ++q) {
            a[q] = b[q] = c[q] = make_ulonglong2(0ull, 0ull);
            if (hb + 32 * q + lane < nh) need |= (j >= 2 ? 7u : j >= 1 ? 3u : 1u) << (3 * q);
          }
          while (true) {
            const unsigned nd = need;
#pragma unroll
            for (int q = 0; q < kStageChunks; ++q) {
              const int h = hb + 32 * q + lane;
              const int jr = h < nh ? hid[h] : 0;
              if (nd & (1u << (3 * q))) a[q] = ld_relaxed_b128(Wp + jr);
              if (nd & (2u << (3 * q))) b[q] = ld_relaxed_b128(Np + jr);
              if (nd & (4u << (3 * q))) c[q] = ld_relaxed_b128(Zp + jr);
            }
#pragma unroll
            for (int q = 0; q < kStageChunks; ++q) {
              if ((nd & (1u << (3 * q))) && tag_ok(a[q], tw)) need &= ~(1u << (3 * q));
              if ((nd & (2u << (3 * q))) && tag_ok(b[q], tw)) need &= ~(2u << (3 * q));
              if ((nd & (4u << (3 * q))) && tag_ok(c[q], tz)) need &= ~(4u << (3 * q));
            }
            if (__all_sync(0xffffffffu, need == 0)) break;
            if ((++spins & 63u) == 0) {
              int give_up = 0;
              if (lane == 0) {
                if (*(volatile int*)timeout || *(volatile int*)&ps.fail) {
                  give_up = 1;
                } else {
                  const unsigned long long now = global_ns();
                  if (t0 == 0) t0 = now;
                  else if ((long long)(now - t0) > d.spin_ns) { atomicExch(timeout, 1); give_up = 1; }
                }
              }
              if (__shfl_sync(0xffffffffu, give_up, 0)) { ok = false; break; }
            }
          }
          if (!ok) break;
#pragma unroll
          for (int q = 0; q < kStageChunks; ++q) {
            const int h = hb + 32 * q + lane;
            if (h < nh) {
              stW[h] = tagged_value(a[q]);
              if (j >= 1) stN[h] = tagged_value(b[q]);
              if (j >= 2) stZ[h] = tagged_value(c[q]);
            }
          }
        }
        if (!ok && lane == 0) ps.fail = 1;
        __syncwarp();
        if (lane == 0) mb_arrive(&ps.mb_stage);
        if (!ok) break;
      }
    } else {
      // ================= compute warps =================
      const int cw = warp - kPipeRoleWarps;
      double alpha_prev = 0.0, beta_prev = 0.0;
      while (true) {
        double* uc = (k & 1) ? uB : uA;    // u_k
        double* up = (k & 1) ? uA : uB;    // u_(k-1), then u_(k+1)
        // (h) of the previous iteration's scalars: z_(k-1), s_(k-1), r_k, u_k, w_k (w_k and z_(k-1) published)
        if (k > 0) {
          ulonglong2* Wn = Wt + (size_t)(k % 3) * n;
          ulonglong2* Zc = Zt + (size_t)((k + 2) % 3) * n;
          const unsigned tw = pipe_tag(pass, k), tz = pipe_tag(pass, k - 1);
          for (int i = ctid; i < nloc; i += nct) {
            const double zi = k == 1 ? nv[i] : fma(beta_prev, z[i], nv[i]);
            const double si = k == 1 ? w[i] : fma(beta_prev, sv[i], w[i]);
            z[i] = zi;
            sv[i] = si;
            const double ri = fma(-alpha_prev, si, r[i]);
            r[i] = ri;
            uc[i] = dil[i] * ri;
            const double wi = fma(-alpha_prev, zi, w[i]);
            w[i] = wi;
            publish(Wn + r0 + i, wi, tw);
            publish(Zc + r0 + i, zi, tz);
          }
        }
        // (a) partial (r,u), (w,u), (r,r) of this warp's rows
        {
          double v3[3] = {0.0, 0.0, 0.0};
          for (int i = ctid; i < nloc; i += nct) {
            const double ui = uc[i], ri = r[i];
            v3[0] += ri * ui;
            v3[1] += w[i] * ui;
            v3[2] += ri * ri;
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int E = (int)__reduce_max_sync(0xffffffffu, (unsigned)fx64_exponent(v3[c]));
            const long long S = warp_sum57(E < fx::kBadExp ? fx64_image(v3[c], E) : 0ll);
            if (lane == 0) {
              ps.ws[c][cw] = S;
              ps.we[c][cw] = E;
            }
          }
          if (lane == 0) mb_arrive(&ps.mb_part);
        }
        // (c) m = D^-1 w: own rows, and the halo from the staged owner values
        bool ok = mb_wait_warp(&ps.mb_stage, (unsigned)(k & 1), timeout, d.spin_ns);
        for (int i = ctid; i < nloc; i += nct) ext[i] = dil[i] * w[i];
        for (int h = ctid; h < nh; h += nct) {
          double wj;
          if (k == 0) {
            wj = stW[h];
          } else {
            const double zj = k == 1 ? stN[h] : fma(beta_prev, stZ[h], stN[h]);
            wj = fma(-alpha_prev, zj, stW[h]);
          }
          ext[nloc + h] = dih[h] * wj;
        }
        __syncwarp();
        if (lane == 0) mb_arrive(&ps.mb_ext);
        ok = mb_wait_warp(&ps.mb_ext, (unsigned)(k & 1), timeout, d.spin_ns) && ok;   // every warp's m
        // (d) n_k = K m, published
        {
          ulonglong2* Nc = Nt + (size_t)(k % 3) * n;
          const unsigned tn = pipe_tag(pass, k);
          const int g = ctid / T, l = ctid % T, ng = nct / T;
          for (int b0 = 0; b0 < nloc; b0 += ng) {
            const int il = b0 + g;
            double sum = 0.0;
            if (il < nloc) {
              const int kk1 = row[il + 1];
              for (int kk = row[il] + l; kk < kk1; kk += T) sum = fma(val[kk], ext[col[kk]], sum);
            }
            if (T > 1) {
#pragma unroll
              for (int o = T / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, T);
            }
            if (il < nloc && l == 0) {
              nv[il] = sum;
              publish(Nc + r0 + il, sum, tn);
            }
          }
        }
        // (f) p_(k-1) = u_(k-1) + beta_(k-1) p_(k-2), x_k = x_(k-1) + alpha_(k-1) p_(k-1)
        if (k > 0) {
          for (int i = ctid; i < nloc; i += nct) {
            const double pi = k == 1 ? up[i] : fma(beta_prev, p[i], up[i]);
            p[i] = pi;
            x[i] = fma(alpha_prev, pi, x[i]);
          }
        }
        // (g) the scalars of iteration k
        ok = mb_wait_warp(&ps.mb_scal, (unsigned)(k & 1), timeout, d.spin_ns) && ok;
        if (!ok) {
          if (lane == 0) ps.fail = 1;
          break;
        }
        const int st = ps.status;
        alpha_prev = ps.alpha;
        beta_prev = ps.beta;
        ++red;
        ++k;
        if (st >= 0) break;
        // the next (h) reads n_k of rows another warp wrote (T > 1), and the next (c) rewrites the
        // product's input: every compute warp has passed (d) and (f) of iteration k - 1
        __syncwarp();
        if (lane == 0) mb_arrive(&ps.mb_end);
        if (!mb_wait_warp(&ps.mb_end, (unsigned)((k - 1) & 1), timeout, d.spin_ns)) {
          if (lane == 0) ps.fail = 1;
          break;
        }
      }
    }
    __syncthreads();
    if (tid == 0) {   // the next pass initialises them again
      mb_inval(&ps.mb_part);
      mb_inval(&ps.mb_ext);
      mb_inval(&ps.mb_end);
      mb_inval(&ps.mb_stage);
      mb_inval(&ps.mb_tot);
      mb_inval(&ps.mb_scal);
    }
    if (ps.fail || ps.status == CGP_ERR_TIMEOUT) return;
    const int st = ps.status;
    if (st != CGP_OK && st != kRestartCode) pending = st;
    its += ps.iter_done;            // iterations whose update ran
    red = red0 + ps.iter_done + 1;  // the same reduction count in every role
    rr_rec = ps.tot[2];
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

template <int T>
__global__ void __launch_bounds__(MAX_BLOCK) pcg_pipe_kernel(Desc d) {
  __shared__ Shared sh;
  mark_pending(d, blockIdx.x);
  solve_fp64_pipe<T>(d, blockIdx.x, sh);
}

template <int T>
__global__ void __launch_bounds__(MAX_BLOCK)
    pcg_pipe_batched_kernel(const Desc* __restrict__ descs, const int* __restrict__ blk_inst,
                            unsigned long long* t_start) {
  __shared__ Shared sh;
  if (t_start && blockIdx.x == 0 && threadIdx.x == 0) *t_start = global_ns();
  const Desc& d = descs[blk_inst[blockIdx.x]];
  const int lb = blockIdx.x - d.blk0;
  mark_pending(d, lb);
  solve_fp64_pipe<T>(d, lb, sh);
}

}  // namespace

const void* pipe_kernel_ptr(int lanes, bool batched) {
  switch (lanes) {
    case 1: return batched ? (const void*)pcg_pipe_batched_kernel<1> : (const void*)pcg_pipe_kernel<1>;
    case 2: return batched ? (const void*)pcg_pipe_batched_kernel<2> : (const void*)pcg_pipe_kernel<2>;
    case 4: return batched ? (const void*)pcg_pipe_batched_kernel<4> : (const void*)pcg_pipe_kernel<4>;
    default: return nullptr;
  }
}

}  // namespace cgp
