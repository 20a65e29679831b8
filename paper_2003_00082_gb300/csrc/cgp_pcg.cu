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

#include "cgp_solver.cuh"

namespace cgp {

// kernels compiled in their own units (cgp_pcg_batch.cu, cgp_pipe.cu)
const void* batched_kernel_ptr(int lanes, bool res);
const void* pipe_kernel_ptr(int lanes, bool batched);

namespace {

template <int T, bool RES>
__global__ void __launch_bounds__(MAX_BLOCK) pcg_persistent_kernel(Desc d) {
  __shared__ Shared sh;
  mark_pending(d, blockIdx.x);
  if (d.mixed)
    solve_mixed<T, RES>(d, blockIdx.x, sh);
  else if (d.classic)
    solve_fp64<T, RES>(d, blockIdx.x, sh);
  else if (RES && d.pipelined && d.stencil)
    solve_fp64_pl<T>(d, blockIdx.x, sh);
  else
    solve_fp64_sr<T, RES>(d, blockIdx.x, sh);
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

using PcgFn = const void*;   // a kernel's address, for launches and occupancy queries

PcgFn pcg_kernel_for(int lanes, bool res) {
  switch (lanes) {
    case 1: return res ? (PcgFn)pcg_persistent_kernel<1, true> : (PcgFn)pcg_persistent_kernel<1, false>;
    case 2: return res ? (PcgFn)pcg_persistent_kernel<2, true> : (PcgFn)pcg_persistent_kernel<2, false>;
    case 4: return res ? (PcgFn)pcg_persistent_kernel<4, true> : (PcgFn)pcg_persistent_kernel<4, false>;
    case 8: return res ? (PcgFn)pcg_persistent_kernel<8, true> : (PcgFn)pcg_persistent_kernel<8, false>;
    case 32: return res ? (PcgFn)pcg_persistent_kernel<32, true> : (PcgFn)pcg_persistent_kernel<32, false>;
    default: return nullptr;
  }
}

using BatchFn = const void*;

BatchFn batched_kernel_for(int lanes, bool res) { return batched_kernel_ptr(lanes, res); }

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
  bool stencil = false;   // resident O-grid tiles with the stencil product
  bool pl = false;        // ... in the pipelined iteration (solve_fp64_pl)
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
//
// tiles != 0 (an O-grid registered with cgp_mesh_set_ogrid): the bisection
// runs on the (angle, ring) indices of the nodes instead of their
// coordinates, so every block owns a near-rectangle of the index grid, and
// the system also carries what the stencil product needs (tile_stencil).
int tile_stencil(cgp_mesh_impl* m, PermSystem& ps, const std::vector<int>& perm, const std::vector<int>& inv,
                 const std::vector<double>& K);

int get_perm_system(cgp_mesh_impl* m, int nblk, PermSystem*& out, int tiles = 0) {
  const int dir = m->far_dirichlet;
  tiles = tiles && m->st_nt > 0;
  for (PermSystem& ps : m->psys)
    if (ps.nblk == nblk && ps.dirichlet == dir && ps.tiles == tiles) {
      out = &ps;
      return CGP_OK;
    }
  const int n = m->n_c, nnz = m->nnz, chunk = (n + nblk - 1) / nblk;
  std::vector<double> xy(2 * (size_t)n), K(nnz), dv(n);
  CGP_CUDA(cudaDeviceSynchronize());
  CGP_CUDA(cudaMemcpy(xy.data(), m->xy_c, xy.size() * 8, cudaMemcpyDeviceToHost));
  if (tiles)
    for (int i = 0; i < n; ++i) {   // (angle index, ring index)
      xy[2 * (size_t)i] = (double)(i % m->st_nt);
      xy[2 * (size_t)i + 1] = (double)(i / m->st_nt);
    }
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
  ps.tiles = tiles;
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
  if (tiles) {
    st = tile_stencil(m, ps, perm, inv, K);
    if (st != CGP_OK) {
      cudaFree(ps.base);
      cudaFree(ps.plan.base);
      return st;
    }
  }
  m->psys.push_back(ps);
  out = &m->psys.back();
  return CGP_OK;
}

// (angle, ring) offset of stencil entry k, as in the standalone stencil product
constexpr int kStencil = 7;
inline int tile_di(int k) { return k == 1 || k == 5 ? 1 : (k == 2 || k == 6 ? -1 : 0); }
inline int tile_dj(int k) { return k == 3 || k == 5 ? 1 : (k == 4 || k == 6 ? -1 : 0); }

// The stencil data of a tiled system: the seven coefficient planes in the
// new row order (from the system's own values, so the far-field variant's
// identity rows come out right), every block's box (its index-grid bounding
// rectangle with a one-node ring), the box position of every row, and every
// block's halo as (box position, row of another block) pairs.  A neighbour
// reached across the periodic angle seam is taken through the halo even when
// the block owns it.
int tile_stencil(cgp_mesh_impl* m, PermSystem& ps, const std::vector<int>& perm, const std::vector<int>& inv,
                 const std::vector<double>& K) {
  const int n = ps.n, nblk = ps.nblk, nt = m->st_nt, chunk = (n + nblk - 1) / nblk;
  std::vector<double> planes((size_t)kStencil * n, 0.0);
  std::vector<int> bpos(n), bdim(nblk), hptr(nblk + 1, 0), hidx, hpos;
  int box_cap = 0, max_halo = 0;
  for (int b = 0; b < nblk; ++b) {
    const int r0 = std::min(n, b * chunk), r1 = std::min(n, r0 + chunk);
    int a0 = 1 << 30, a1 = -1, j0 = 1 << 30, j1 = -1;
    for (int r = r0; r < r1; ++r) {
      const int o = perm[r], i = o % nt, j = o / nt;
      a0 = std::min(a0, i); a1 = std::max(a1, i); j0 = std::min(j0, j); j1 = std::max(j1, j);
    }
    const int Ba = r1 > r0 ? a1 - a0 + 3 : 1, Bb = r1 > r0 ? j1 - j0 + 3 : 1;
    bdim[b] = Ba;
    box_cap = std::max(box_cap, Ba * Bb);
    std::vector<std::pair<int, int>> halo;   // (box position, row)
    for (int r = r0; r < r1; ++r) {
      const int o = perm[r], i = o % nt, j = o / nt;
      bpos[r] = (j - j0 + 1) * Ba + (i - a0 + 1);
    }
    for (int r = r0; r < r1; ++r) {
      const int o = perm[r], i = o % nt, j = o / nt;
      for (int k = m->h_rowptr[o]; k < m->h_rowptr[o + 1]; ++k) {
        const int c = m->h_col[k], ic = c % nt, jc = c / nt;
        int di = ic - i;
        if (di > 1) di -= nt;
        if (di < -1) di += nt;
        const int dj = jc - j;
        int dir = -1;
        for (int q = 0; q < kStencil; ++q)
          if (tile_di(q) == di && tile_dj(q) == dj) dir = q;
        if (dir < 0) return fail(CGP_ERR_INVALID_ARG, "O-grid tiles: a row's pattern is not the seven-point stencil");
        planes[(size_t)dir * n + r] = K[k];
        const int p = bpos[r] + dj * Ba + di, q = inv[c];
        if (q >= r0 && q < r1 && bpos[q] == p) continue;   // owned, at its own box position
        halo.push_back({p, q});
      }
    }
    std::sort(halo.begin(), halo.end());
    halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
    for (size_t t = 1; t < halo.size(); ++t)
      if (halo[t].first == halo[t - 1].first)
        return fail(CGP_ERR_INVALID_ARG, "O-grid tiles: two rows at one box position");
    for (const auto& hq : halo) {
      hpos.push_back(hq.first);
      hidx.push_back(hq.second);
    }
    hptr[b + 1] = hptr[b] + (int)halo.size();
    max_halo = std::max(max_halo, (int)halo.size());
  }
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t nh = std::max<size_t>(1, hidx.size());
  const size_t o_pl = 0, o_bp = o_pl + al((size_t)kStencil * n * 8), o_bd = o_bp + al((size_t)n * 4),
               o_hp = o_bd + al((size_t)nblk * 4), o_hi = o_hp + al((size_t)(nblk + 1) * 4),
               o_hs = o_hi + al(nh * 4), bytes = o_hs + al(nh * 4);
  void* base = nullptr;
  CGP_CUDA(cudaMalloc(&base, bytes));
  char* c = static_cast<char*>(base);
  ps.st_base = base;
  ps.planes = (double*)(c + o_pl);
  ps.bpos = (int*)(c + o_bp);
  ps.bdim = (int*)(c + o_bd);
  ps.st_hptr = (int*)(c + o_hp);
  ps.st_hidx = (int*)(c + o_hi);
  ps.st_hpos = (int*)(c + o_hs);
  ps.box_cap = box_cap;
  ps.st_max_halo = max_halo;
  cudaError_t e = cudaMemcpy(ps.planes, planes.data(), planes.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ps.bpos, bpos.data(), (size_t)n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ps.bdim, bdim.data(), (size_t)nblk * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ps.st_hptr, hptr.data(), (size_t)(nblk + 1) * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !hidx.empty()) e = cudaMemcpy(ps.st_hidx, hidx.data(), hidx.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !hpos.empty()) e = cudaMemcpy(ps.st_hpos, hpos.data(), hpos.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(base);
    ps.st_base = nullptr;
    return cuda_fail(e, "cudaMemcpy(O-grid tiles)");
  }
  return CGP_OK;
}

// Solver variants of one launch.
enum SolverKind { KIND_FP64_CLASSIC = 0, KIND_MIXED = 1, KIND_FP64_SR = 2, KIND_FP64_PIPE = 3 };

SolverKind solver_kind(bool mixed, int flags) {
  if (mixed) return KIND_MIXED;
  if (flags & 2) return KIND_FP64_CLASSIC;
  return (flags & 16) ? KIND_FP64_PIPE : KIND_FP64_SR;
}

// Kernel of a resident launch of this kind: the pipelined iteration has
// kernels of its own for 1, 2 or 4 lanes per row and at least 256 threads
// per block (four warps of a block are given to its reductions and its grid
// barrier); otherwise, or when rows are not resident, a pipelined request
// runs the single-reduction form.
constexpr int kPipeMinBlock = 256;
PcgFn resident_kernel_for(SolverKind& kind, int lanes, int block) {
  if (kind == KIND_FP64_PIPE) {
    if (block >= kPipeMinBlock)
      if (PcgFn f = pipe_kernel_ptr(lanes, false)) return f;
    kind = KIND_FP64_SR;
  }
  return pcg_kernel_for(lanes, true);
}

BatchFn resident_batched_kernel_for(SolverKind& kind, int lanes, int block) {
  if (kind == KIND_FP64_PIPE) {
    if (block >= kPipeMinBlock)
      if (BatchFn f = pipe_kernel_ptr(lanes, true)) return f;
    kind = KIND_FP64_SR;
  }
  return batched_kernel_for(lanes, true);
}

// Dynamic shared memory of a block that keeps its rows resident: the classic
// FP64 solver needs seven vectors, the halo buffer and an FP64 CSR slice; the
// single-reduction FP64 solver nine vectors, the halo buffer, D^-1 of the
// halo, three staging buffers of the halo and the slice; the pipelined FP64
// solver eleven vectors, the halo buffer, D^-1 of the halo, three staging
// buffers and the slice; the mixed solver six
// FP32 vectors, D^-1, the halo buffer, D^-1 of the halo, three staging
// buffers and an FP32 slice.
size_t res_smem_bytes(SolverKind kind, int chunk, const HaloPlan& hp) {
  const size_t ints = 4 * ((size_t)chunk + 1 + hp.max_nnz + hp.max_halo);
  size_t s = 0;
  if (kind == KIND_MIXED)
    s = 4 * ((size_t)9 * chunk + 6 * (size_t)hp.max_halo + 2 * (size_t)hp.max_nnz + 1);
  else if (kind == KIND_FP64_CLASSIC)
    s = 8 * ((size_t)7 * chunk + hp.max_halo + hp.max_nnz) + ints;
  else if (kind == KIND_FP64_PIPE)
    s = 8 * ((size_t)12 * chunk + 5 * (size_t)hp.max_halo + hp.max_nnz) + ints;
  else
    s = 8 * ((size_t)10 * chunk + 5 * (size_t)hp.max_halo + hp.max_nnz) + ints;
  return (s + 15) / 16 * 16;
}

// Shared memory a resident block needs for its chunk and CSR slice, before
// the halo is known (the lower bound the planners size chunks by).
size_t res_smem_rows(SolverKind kind, int chunk, int nnz) {
  HaloPlan none;
  none.max_nnz = nnz;
  return res_smem_bytes(kind, chunk, none);
}

// Dynamic shared memory of a resident single-reduction FP64 block on O-grid
// tiles: nine vectors, the padded box, D^-1 of the halo, seven coefficient
// planes, three staging buffers of the halo; box positions of the rows and
// the halo, and the halo's global rows.
size_t res_smem_stencil(int chunk, int max_halo, int box_cap) {
  const size_t s = 8 * ((size_t)16 * chunk + (size_t)box_cap + 4 * (size_t)max_halo) +
                   4 * ((size_t)chunk + 2 * (size_t)max_halo);
  return (s + 15) / 16 * 16;
}

// The same for the pipelined iteration on the tiles (solve_fp64_pl): eleven
// vectors, the padded box, D^-1 of the halo and the seven planes; box
// positions and product order of the rows, box positions and global rows of
// the halo.
size_t res_smem_stencil_pl(int chunk, int max_halo, int box_cap) {
  const size_t s = 8 * ((size_t)18 * chunk + (size_t)box_cap + (size_t)max_halo) +
                   4 * (2 * (size_t)chunk + 2 * (size_t)max_halo);
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
  // tuning flag bit 2: rows renumbered by coordinate bisection (compact chunks, smaller halos);
  // bit 5 (FP64 single-reduction or pipelined form on a registered O-grid): rows renumbered into
  // index-grid tiles, whose resident product uses the seven-point stencil
  const bool tiles = m && (tu.flags & 32) && !mixed && !(tu.flags & 2) && m->st_nt > 0;
  PermSystem* ps = nullptr;
  if (m && ((tu.flags & 4) || tiles)) {
    int st = get_perm_system(m, nblk, ps, tiles ? 1 : 0);
    if (st != CGP_OK) return st;
    out.halo = ps->plan;   // the non-resident path reads the permuted pattern directly
  }
  if (ps_out) *ps_out = ps;
  if (!m || (tu.flags & 1)) return CGP_OK;
  if (tiles) {
    const int chunk = (n + nblk - 1) / nblk;
    PcgFn fnr = pcg_kernel_for(lanes, true);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, (const void*)fnr) != cudaSuccess) {
      cudaGetLastError();
      return CGP_OK;
    }
    const size_t limit = (size_t)std::max(0, optin_smem(device) - (int)fa.sharedSizeBytes - 1024);
    // bit 4 with the tiles: the pipelined iteration, given three polling warps and five computing ones
    const bool pl = (tu.flags & 16) && block >= 256 && nblk <= 2048;
    const size_t smem = pl ? res_smem_stencil_pl(chunk, ps->st_max_halo, ps->box_cap)
                           : res_smem_stencil(chunk, ps->st_max_halo, ps->box_cap);
    if (smem > limit) return CGP_OK;
    if (cudaFuncSetAttribute((const void*)fnr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return CGP_OK;
    }
    if (coresident_blocks(fnr, block, device, smem) < nblk) return CGP_OK;
    out.fn = fnr;
    out.smem = smem;
    out.halo_cap = ps->st_max_halo;
    out.res = true;
    out.stencil = true;
    out.pl = pl;
    return CGP_OK;
  }
  const int chunk = (n + nblk - 1) / nblk;
  const std::vector<int>& hrp = ps ? ps->h_rowptr : m->h_rowptr;
  // rough size check before building a plan
  const int rough_nnz = hrp[std::min(n, chunk)] - hrp[0];
  SolverKind kind = solver_kind(mixed, tu.flags);
  PcgFn fnr = resident_kernel_for(kind, lanes, block);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, (const void*)fnr) != cudaSuccess) {
    cudaGetLastError();
    return CGP_OK;
  }
  const size_t limit = (size_t)std::max(0, optin_smem(device) - (int)fa.sharedSizeBytes - 1024);
  if (res_smem_rows(kind, chunk, rough_nnz) > limit) return CGP_OK;
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
  d.pipelined = (flags & 16) ? 1 : 0;
  d.tagged = (flags & 24) ? 1 : 0;   // the pipelined iteration reads its reductions from tagged slots
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
    if (plan.stencil) {   // the tiles' own halo lists and the stencil data
      d.stencil = 1;
      d.box_cap = ps->box_cap;
      d.planes = ps->planes;
      d.bpos = ps->bpos;
      d.bdim = ps->bdim;
      d.hptr = ps->st_hptr;
      d.hidx = ps->st_hidx;
      d.hpos = ps->st_hpos;
      d.pipelined = plan.pl ? 1 : 0;
      d.nflag = m->nflag;
    }
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
  SolverKind kind = solver_kind(mixed, sh.flags);
  bool res = !(sh.flags & 1);
  size_t smem = 0;
  BatchFn fnr = resident_batched_kernel_for(kind, lanes, block);
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
    if (res_smem_rows(kind, chunk, rough_nnz) > limit) {
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

// Wave schedule: every instance gets about rows_per_block rows per block
// (256 << (flags bits 5-6): 256 as a solve of it alone would use, up to 2048),
// at most one SM's worth of blocks and at least as many blocks as keep its
// chunk in shared memory; instances are packed largest first into waves of
// at most blocks_per_sm x SMs blocks, and the waves run as consecutive
// cooperative launches, the wave of the smallest instances first.  Small
// instances then share the GPU, and a large one gets all of it (256 rows a
// block) or shares it with others of its size (more rows a block: the
// iteration is bound by the latency of its reductions, not by its rows).
int batch_plan_waves(cgp_batch_s* B, const BatchShape& sh, const cgp_solve_opts& o) {
  const int lanes = sh.lanes > 0 ? sh.lanes : 1;
  const int block = sh.block > 0 ? sh.block : 512;
  const bool mixed = o.precision == CGP_MIXED;
  BatchFn fn0 = batched_kernel_for(lanes, false);
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
  SolverKind kind = solver_kind(mixed, sh.flags);
  BatchFn fnr = resident_batched_kernel_for(kind, lanes, block);
  cudaFuncAttributes fa{};
  bool can_res = !(sh.flags & 1) && cudaFuncGetAttributes(&fa, (const void*)fnr) == cudaSuccess;
  if (!can_res) cudaGetLastError();
  const size_t limit = can_res ? (size_t)std::max(0, optin_smem(B->device) - (int)fa.sharedSizeBytes - 1024) : 0;
  const int rows = 256 << ((sh.flags >> 5) & 3);
  std::vector<int> nb(count), order(count);
  for (int i = 0; i < count; ++i) {
    const cgp_mesh_impl* m = B->meshes[i];
    const int n = m->n_c;
    int want = (n + rows - 1) / rows;
    if (can_res && rows > 256) {
      // the largest chunk whose rows leave a quarter of the shared memory to the halo
      const int per_row = std::max(1, (m->nnz + n - 1) / std::max(1, n));
      int c = std::min(n, rows);
      while (c > 256 && res_smem_rows(kind, c, c * per_row) * 5 > limit * 4) c -= 64;
      want = std::max(want, (n + c - 1) / c);
    }
    nb[i] = std::max(1, std::min(std::min(cap, m->max_blocks), want));
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
  // the wave whose largest instance is smallest runs first, so the small
  // instances finish early (the order changes the latencies, not the total)
  auto span = [&](const std::vector<int>& grp) {
    double w = 0.0;
    for (int i : grp) {
      const cgp_mesh_impl* m = B->meshes[i];
      w = std::max(w, (double)m->nnz * std::sqrt((double)m->n_c) / nb[i]);
    }
    return w;
  };
  std::stable_sort(groups.begin(), groups.end(),
                   [&](const std::vector<int>& a, const std::vector<int>& b) { return span(a) < span(b); });
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
      if (res_smem_rows(kind, chunk, rough_nnz) > limit) {
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
  if (!valid_shape(what, block, lanes) || blocks < 0 || (flags & ~63))
    return fail(CGP_ERR_INVALID_ARG, "cgp_set_tuning: block must be 0 or a multiple of 32 in [64, 512] "
                                     "(solver) or [64, 256] (SpMV), "
                                     "lanes 0, 1, 2, 4, 8 or 32, blocks >= 0, flags 0 to 63");
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
  if (!valid_shape(CGP_TUNE_SOLVE_FP64, block, lanes) || blocks_per_sm < 0 || (flags & ~127))
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
  const int rows[3] = {0, 2, 3};   // waves: 256, 1024 or 2048 rows a block (flags bits 5-6)
  // iteration flags: rows in global memory (bit 0), tagged reductions (bit 3), and for FP64 the textbook form (bit 1)
  const int mixed_fl[3] = {0, 1, 8}, fp64_fl[6] = {0, 1, 2, 3, 8, 9};
  const bool mixed_b = batch->opts.precision == CGP_MIXED;
  const int* base_fl = mixed_b ? mixed_fl : fp64_fl;
  const int nflags = mixed_b ? 3 : 6;
  for (int fl = 0; fl < 2 * nflags; ++fl)   // bit 2 (one packed launch instead of waves) on top
    for (int rw : rows)
      for (int bk : blocks)
        for (int ln : lanes)
          for (int ps : per_sm) {
            if (rw && (fl >= nflags || ps > 1)) continue;   // more rows a block: waves, one block per SM
            BatchShape cand{bk, ln, ps, base_fl[fl % nflags] | (fl >= nflags ? 4 : 0) | (rw << 5)};
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
  // bit 1 (classic FP64 iteration), bit 4 (pipelined iteration, rows
  // resident, reductions always tagged) and bit 5 (O-grid tiles with the
  // stencil product, single-reduction form, registered O-grids only) only
  // for FP64; bit 2 (bisection order) and bit 3 (tagged reductions: of the
  // single-reduction form, or of the FP32 inner iterations) for both
  std::vector<int> flag_set;
  for (int fl = 0; fl < 64; ++fl) {
    if (precision == CGP_MIXED && (fl & 50)) continue;   // mixed: bits 0, 2 and 3
    if ((fl & 2) && (fl & 8)) continue;
    if ((fl & 16) && (fl & 11)) continue;
    if ((fl & 32) && ((fl & 7) || m->st_nt <= 0)) continue;
    // the pipelined iteration on the tiles (bits 4 and 5) ties the single-reduction tiles from x0 = 0
    // and loses its margin to the restart from the true residual on warm starts: not a candidate
    if ((fl & 48) == 48) continue;
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
