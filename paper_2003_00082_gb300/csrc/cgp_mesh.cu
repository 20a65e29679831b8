// Mesh pair construction and Galerkin P1 assembly (Sect. 2.3 of the paper).
//
// The host builds the integer structure: the coarse edge table (sorted by
// (min vertex, max vertex)), the fine numbering of the uniform 4-way split
// (Eq. 18 with k = 1), the CSR pattern of K (node graph plus diagonal,
// columns ascending) and the node -> triangle incidence lists.  The GPU
// computes every floating-point value: fine-node coordinates, K, Gx, Gy and
// the Jacobi inverse diagonal.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>

#include "cgp_internal.h"

namespace cgp {

static thread_local std::string g_last_error;

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(e == cudaErrorMemoryAllocation ? CGP_ERR_OOM : CGP_ERR_CUDA, m);
}

namespace {

// ---------------------------------------------------------------------------
// per-row assembly: row i gathers the contributions of its incident
// triangles in increasing triangle order (deterministic).  On triangle T with
// b_m = y_{m+1} - y_{m+2}, c_m = x_{m+2} - x_{m+1} and twice its area a2:
//   K_T[l][m]  = (b_l b_m + c_l c_m) / (2 a2)      (= A grad psi_l . grad psi_m)
//   Gx_T[l][m] = b_l / 6,  Gy_T[l][m] = c_l / 6    (= int_T psi_m d_x psi_l)
// Products and sums are rounded separately (no contraction) so the values
// do not depend on the compiler's FMA choices.
// ---------------------------------------------------------------------------
__global__ void assemble_values_kernel(int n, const int* __restrict__ rowptr,
                                       const int* __restrict__ col,
                                       const int* __restrict__ inc_ptr,
                                       const int* __restrict__ inc_tri,
                                       const int* __restrict__ tri,
                                       const double2* __restrict__ xy, double* __restrict__ K,
                                       double* __restrict__ Gx, double* __restrict__ Gy,
                                       double* __restrict__ dinv, float* __restrict__ K32,
                                       float* __restrict__ dinv32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k0 = rowptr[i], k1 = rowptr[i + 1];
  for (int k = k0; k < k1; ++k) { K[k] = 0.0; Gx[k] = 0.0; Gy[k] = 0.0; }
  for (int s = inc_ptr[i]; s < inc_ptr[i + 1]; ++s) {
    const int code = inc_tri[s];
    const int t = code >> 2, l = code & 3;
    const int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
    double x[3], y[3];
    for (int m = 0; m < 3; ++m) { double2 p = xy[v[m]]; x[m] = p.x; y[m] = p.y; }
    double b[3], c[3];
    for (int m = 0; m < 3; ++m) {
      b[m] = __dsub_rn(y[(m + 1) % 3], y[(m + 2) % 3]);
      c[m] = __dsub_rn(x[(m + 2) % 3], x[(m + 1) % 3]);
    }
    const double a2 = __dsub_rn(__dmul_rn(__dsub_rn(x[1], x[0]), __dsub_rn(y[2], y[0])),
                                __dmul_rn(__dsub_rn(x[2], x[0]), __dsub_rn(y[1], y[0])));
    const double den = __dmul_rn(2.0, a2);
    const double gxl = b[l] / 6.0, gyl = c[l] / 6.0;
    for (int m = 0; m < 3; ++m) {
      int pos = k0;
      while (pos < k1 && col[pos] != v[m]) ++pos;
      if (pos == k1) continue;  // cannot happen for a pattern built from the same triangles
      const double kv = __dadd_rn(__dmul_rn(b[l], b[m]), __dmul_rn(c[l], c[m])) / den;
      K[pos] = __dadd_rn(K[pos], kv);
      Gx[pos] = __dadd_rn(Gx[pos], gxl);
      Gy[pos] = __dadd_rn(Gy[pos], gyl);
    }
  }
  double diag = 0.0;
  for (int k = k0; k < k1; ++k) {
    K32[k] = (float)K[k];
    if (col[k] == i) diag = K[k];
  }
  const double di = 1.0 / diag;
  dinv[i] = di;
  dinv32[i] = (float)di;
}

// fine node coordinates: coarse nodes first, then edge midpoints (x_a + x_b) / 2
__global__ void fine_coords_kernel(int n_c, int n_e, const double2* __restrict__ xy_c,
                                   const int2* __restrict__ edges, double2* __restrict__ xy_f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_c) {
    xy_f[i] = xy_c[i];
  } else if (i < n_c + n_e) {
    int2 e = edges[i - n_c];
    double2 a = xy_c[e.x], b = xy_c[e.y];
    xy_f[i] = make_double2(__dmul_rn(__dadd_rn(a.x, b.x), 0.5), __dmul_rn(__dadd_rn(a.y, b.y), 0.5));
  }
}

// midpoints of level-l edges: node n_l + e of level l + 1 sits at (x_a + x_b) / 2
__global__ void fine_coords_level_kernel(int n_l, int e_l, const int2* __restrict__ edges, double2* __restrict__ xy_f) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= e_l) return;
  const int2 ed = edges[e];
  const double2 a = xy_f[ed.x], b = xy_f[ed.y];
  xy_f[n_l + e] = make_double2(__dmul_rn(__dadd_rn(a.x, b.x), 0.5), __dmul_rn(__dadd_rn(a.y, b.y), 0.5));
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Edges of one level: (min, max) vertex pairs sorted lexicographically; side k
// of triangle t (vertices k, k+1) gets edge id tri_edge[3 t + k].
void level_edges(const std::vector<int>& tri, int n_l, std::vector<int>& edges, std::vector<int>& tri_edge) {
  const size_t t_l = tri.size() / 3;
  std::vector<std::pair<long long, int>> keys(3 * t_l);
  for (size_t t = 0; t < t_l; ++t)
    for (int k = 0; k < 3; ++k) {
      const int a = tri[3 * t + k], b = tri[3 * t + (k + 1) % 3];
      const int lo = std::min(a, b), hi = std::max(a, b);
      keys[3 * t + k] = {(long long)lo * n_l + hi, (int)(3 * t + k)};
    }
  std::sort(keys.begin(), keys.end());
  tri_edge.assign(3 * t_l, 0);
  edges.clear();
  int ne = -1;
  long long prev = -1;
  for (auto& kv : keys) {
    if (kv.first != prev) {
      ++ne;
      prev = kv.first;
      edges.push_back((int)(kv.first / n_l));
      edges.push_back((int)(kv.first % n_l));
    }
    tri_edge[kv.second] = ne;
  }
}

}  // namespace

int launch_assemble_values(cgp_mesh_impl* m, cudaStream_t s) {
  const int bs = 128;
  assemble_values_kernel<<<(m->n_c + bs - 1) / bs, bs, 0, s>>>(
      m->n_c, m->rowptr, m->col, m->inc_ptr, m->inc_tri, m->tri_c,
      reinterpret_cast<const double2*>(m->xy_c), m->K, m->Gx, m->Gy, m->dinv, m->K32, m->dinv32);
  CGP_CUDA(cudaGetLastError());
  const int n1 = m->n_c + m->n_e;
  fine_coords_kernel<<<(n1 + 255) / 256, 256, 0, s>>>(
      m->n_c, m->n_e, reinterpret_cast<const double2*>(m->xy_c),
      reinterpret_cast<const int2*>(m->edges), reinterpret_cast<double2*>(m->xy_f));
  CGP_CUDA(cudaGetLastError());
  for (int l = 1; l < m->levels; ++l) {
    const int e_l = m->h_lvl_eoff[l + 1] - m->h_lvl_eoff[l];
    fine_coords_level_kernel<<<(e_l + 255) / 256, 256, 0, s>>>(
        m->h_lvl_nodes[l], e_l, reinterpret_cast<const int2*>(m->edges) + m->h_lvl_eoff[l],
        reinterpret_cast<double2*>(m->xy_f));
    CGP_CUDA(cudaGetLastError());
  }
  return CGP_OK;
}

}  // namespace cgp

using namespace cgp;

extern "C" const char* cgp_last_error(void) { return g_last_error.c_str(); }

extern "C" int cgp_assemble(const double* xy_c, int n_c, const int* tri_c, int t_c, int levels,
                            cgp_mesh* out) {
  if (!out) return fail(CGP_ERR_INVALID_ARG, "cgp_assemble: out is NULL");
  *out = nullptr;
  if (!xy_c || !tri_c) return fail(CGP_ERR_INVALID_ARG, "cgp_assemble: NULL input");
  if (n_c < 3 || t_c < 1) return fail(CGP_ERR_INVALID_ARG, "cgp_assemble: need n_c >= 3 and t_c >= 1");
  if (levels < 1 || levels > 3) return fail(CGP_ERR_INVALID_ARG, "cgp_assemble: levels must be 1, 2 or 3");
  {
    // every level: t_(l+1) = 4 t_l and n_(l+1) <= n_l + 3 t_l
    long long t = t_c, nn = n_c;
    for (int l = 0; l < levels; ++l) {
      nn += 3 * t;
      t *= 4;
    }
    if (3 * t > (1LL << 30) || nn > (1LL << 30))
      return fail(CGP_ERR_INVALID_ARG, "cgp_assemble: mesh too large for 32-bit indexing");
  }

  // ---- validate triangles ----
  std::vector<int> used(n_c, 0);
  for (int t = 0; t < t_c; ++t) {
    int a = tri_c[3 * t], b = tri_c[3 * t + 1], c = tri_c[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= n_c || b >= n_c || c >= n_c)
      return fail(CGP_ERR_INVALID_ARG, "cgp_assemble: triangle " + std::to_string(t) + " has an index out of range");
    if (a == b || b == c || a == c)
      return fail(CGP_ERR_INVALID_ARG, "cgp_assemble: triangle " + std::to_string(t) + " repeats a vertex");
    double x0 = xy_c[2 * a], y0 = xy_c[2 * a + 1], x1 = xy_c[2 * b], y1 = xy_c[2 * b + 1];
    double x2 = xy_c[2 * c], y2 = xy_c[2 * c + 1];
    double a2 = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
    if (!(a2 > 0.0))
      return fail(CGP_ERR_INVALID_ARG, "cgp_assemble: triangle " + std::to_string(t) + " is clockwise or degenerate");
    used[a] = used[b] = used[c] = 1;
  }
  for (int i = 0; i < n_c; ++i)
    if (!used[i]) return fail(CGP_ERR_INVALID_ARG, "cgp_assemble: node " + std::to_string(i) + " belongs to no triangle");

  int device = 0;
  CGP_CUDA(cudaGetDevice(&device));
  cgp_mesh_s* m = new cgp_mesh_s();
  m->n_c = n_c;
  m->t_c = t_c;
  m->device = device;

  // ---- the nested levels (Eq. 18): each a 4-way split of the previous ----
  // Level l + 1 numbers level l's nodes first, then the midpoints of level l's
  // edges in edge order; child 4 t + c of triangle (a, b, c) with midpoints
  // m_ab, m_bc, m_ca is (a, m_ab, m_ca), (m_ab, b, m_bc), (m_ca, m_bc, c),
  // (m_ab, m_bc, m_ca).  The coarse nodes stay the prefix of every level.
  m->levels = levels;
  m->h_tri_c.assign(tri_c, tri_c + 3 * (size_t)t_c);
  std::vector<int> all_edges, tri_edge, lvl_edges;
  std::vector<int> lvl_tri(m->h_tri_c);
  m->h_lvl_nodes.assign(1, n_c);
  m->h_lvl_eoff.assign(1, 0);
  for (int l = 0; l < levels; ++l) {
    const int n_l = m->h_lvl_nodes[l];
    level_edges(lvl_tri, n_l, lvl_edges, tri_edge);
    const int e_l = (int)(lvl_edges.size() / 2);
    if (l == 0) {
      m->h_edges = lvl_edges;
      m->n_e = e_l;
      m->h_tri_mid.resize(3 * (size_t)t_c);
      for (size_t q = 0; q < 3 * (size_t)t_c; ++q) m->h_tri_mid[q] = n_c + tri_edge[q];
    }
    all_edges.insert(all_edges.end(), lvl_edges.begin(), lvl_edges.end());
    m->h_lvl_eoff.push_back(m->h_lvl_eoff.back() + e_l);
    m->h_lvl_nodes.push_back(n_l + e_l);
    const size_t t_l = lvl_tri.size() / 3;
    if (l + 1 < levels) {   // the next level's triangles
      std::vector<int> next(12 * t_l);
      for (size_t t = 0; t < t_l; ++t) {
        const int a = lvl_tri[3 * t], b = lvl_tri[3 * t + 1], c = lvl_tri[3 * t + 2];
        const int mab = n_l + tri_edge[3 * t], mbc = n_l + tri_edge[3 * t + 1], mca = n_l + tri_edge[3 * t + 2];
        const int ch[12] = {a, mab, mca, mab, b, mbc, mca, mbc, c, mab, mbc, mca};
        std::memcpy(&next[12 * t], ch, sizeof(ch));
      }
      lvl_tri.swap(next);
    } else {                // the fine triangles' parents and their midpoints
      m->t_par = (int)t_l;
      if (levels >= 2) {
        m->h_tri_par = lvl_tri;
        m->h_mid_par.resize(3 * t_l);
        for (size_t q = 0; q < 3 * t_l; ++q) m->h_mid_par[q] = n_l + tri_edge[q];
      }
    }
  }
  m->n_f = m->h_lvl_nodes[levels];
  m->t_f = 4 * m->t_par;

  // ---- CSR pattern of the node graph plus the diagonal ----
  std::vector<int> deg(n_c, 1);
  for (int e = 0; e < m->n_e; ++e) { deg[m->h_edges[2 * e]]++; deg[m->h_edges[2 * e + 1]]++; }
  m->h_rowptr.assign(n_c + 1, 0);
  for (int i = 0; i < n_c; ++i) m->h_rowptr[i + 1] = m->h_rowptr[i] + deg[i];
  m->nnz = m->h_rowptr[n_c];
  m->h_col.assign(m->nnz, 0);
  std::vector<int> fill(m->h_rowptr.begin(), m->h_rowptr.end() - 1);
  for (int i = 0; i < n_c; ++i) m->h_col[fill[i]++] = i;
  for (int e = 0; e < m->n_e; ++e) {
    int a = m->h_edges[2 * e], b = m->h_edges[2 * e + 1];
    m->h_col[fill[a]++] = b;
    m->h_col[fill[b]++] = a;
  }
  for (int i = 0; i < n_c; ++i) std::sort(m->h_col.begin() + m->h_rowptr[i], m->h_col.begin() + m->h_rowptr[i + 1]);

  // ---- node -> incident triangles (triangle * 4 + local vertex), triangle order ----
  std::vector<int> inc_ptr(n_c + 1, 0), inc(3 * (size_t)t_c);
  for (size_t s = 0; s < 3 * (size_t)t_c; ++s) inc_ptr[tri_c[s] + 1]++;
  for (int i = 0; i < n_c; ++i) inc_ptr[i + 1] += inc_ptr[i];
  std::vector<int> ifill(inc_ptr.begin(), inc_ptr.end() - 1);
  for (int t = 0; t < t_c; ++t)
    for (int l = 0; l < 3; ++l) inc[ifill[tri_c[3 * t + l]]++] = t * 4 + l;

  // ---- one device allocation ----
  m->max_blocks = solver_max_blocks(m->device);
  const size_t n = n_c, nz = m->nnz, A = 256;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, A); return o; };
  size_t o_rowptr = take((n + 1) * 4), o_col = take(nz * 4), o_K = take(nz * 8), o_Gx = take(nz * 8),
         o_Gy = take(nz * 8), o_dinv = take(n * 8), o_K32 = take(nz * 4), o_d32i = take(n * 4),
         o_tri = take(3 * (size_t)t_c * 4), o_mid = take(3 * (size_t)t_c * 4),
         o_edges = take(2 * (size_t)m->h_lvl_eoff[levels] * 4), o_tpar = take(m->h_tri_par.size() * 4),
         o_mpar = take(m->h_mid_par.size() * 4), o_xyf = take(2 * (size_t)m->n_f * 8),
         o_xyc = take(2 * n * 8), o_incp = take((n + 1) * 4), o_inc = take(3 * (size_t)t_c * 4),
         o_bp = take(n * 8), o_r = take(n * 8), o_z = take(n * 8), o_p = take(n * 8), o_p2 = take(n * 8), o_q = take(n * 8),
         o_pub64 = take(18 * n * 8), o_f32pub = take(6 * n * 4), o_f32own = take(6 * n * 4),
         o_fpart = take((size_t)m->max_blocks * 8 * 4), o_part = take((size_t)m->max_blocks * 32 * 8),
         o_tpart = take((size_t)m->max_blocks * 6 * 16), o_nflag = take((size_t)m->max_blocks * 4),
         o_bar = take(256),
         o_res = take(sizeof(SolveResult));
  m->d_bytes = off;
  cudaError_t e = cudaMalloc(&m->d_base, m->d_bytes);
  if (e != cudaSuccess) { delete m; return cuda_fail(e, "cudaMalloc(mesh)"); }
  char* base = static_cast<char*>(m->d_base);
  m->rowptr = (int*)(base + o_rowptr);
  m->col = (int*)(base + o_col);
  m->K = (double*)(base + o_K);
  m->Gx = (double*)(base + o_Gx);
  m->Gy = (double*)(base + o_Gy);
  m->dinv = (double*)(base + o_dinv);
  m->K32 = (float*)(base + o_K32);
  m->dinv32 = (float*)(base + o_d32i);
  m->tri_c = (int*)(base + o_tri);
  m->tri_mid = (int*)(base + o_mid);
  m->edges = (int*)(base + o_edges);
  m->tri_par = levels >= 2 ? (int*)(base + o_tpar) : m->tri_c;
  m->mid_par = levels >= 2 ? (int*)(base + o_mpar) : m->tri_mid;
  m->xy_f = (double*)(base + o_xyf);
  m->xy_c = (double*)(base + o_xyc);
  m->inc_ptr = (int*)(base + o_incp);
  m->inc_tri = (int*)(base + o_inc);
  m->bp = (double*)(base + o_bp);
  m->r = (double*)(base + o_r);
  m->z = (double*)(base + o_z);
  m->p = (double*)(base + o_p);
  m->p2 = (double*)(base + o_p2);
  m->q = (double*)(base + o_q);
  m->pub64 = (double*)(base + o_pub64);
  m->f32pub = (float*)(base + o_f32pub);
  m->f32own = (float*)(base + o_f32own);
  m->fpart = (float*)(base + o_fpart);
  m->part = (double*)(base + o_part);
  m->tpart = (unsigned long long*)(base + o_tpart);
  m->nflag = (unsigned*)(base + o_nflag);
  m->bar = (unsigned*)(base + o_bar);
  m->res = (SolveResult*)(base + o_res);
  e = cudaMallocHost(&m->h_res, sizeof(SolveResult));
  if (e != cudaSuccess) { cudaFree(m->d_base); delete m; return cuda_fail(e, "cudaMallocHost(result)"); }

  auto cleanup_fail = [&](int st) { cgp_mesh_destroy(m); return st; };
  auto up = [&](void* dst, const void* src, size_t bytes) -> int {
    cudaError_t ee = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    return ee == cudaSuccess ? CGP_OK : cuda_fail(ee, "cudaMemcpy(assemble)");
  };
  int st = CGP_OK;
  if ((st = up(m->rowptr, m->h_rowptr.data(), (n + 1) * 4)) ||
      (st = up(m->col, m->h_col.data(), nz * 4)) ||
      (st = up(m->tri_c, m->h_tri_c.data(), 3 * (size_t)t_c * 4)) ||
      (st = up(m->tri_mid, m->h_tri_mid.data(), 3 * (size_t)t_c * 4)) ||
      (st = up(m->edges, all_edges.data(), all_edges.size() * 4)) ||
      (levels >= 2 && (st = up(m->tri_par, m->h_tri_par.data(), m->h_tri_par.size() * 4))) ||
      (levels >= 2 && (st = up(m->mid_par, m->h_mid_par.data(), m->h_mid_par.size() * 4))) ||
      (st = up(m->xy_c, xy_c, 2 * n * 8)) || (st = up(m->inc_ptr, inc_ptr.data(), (n + 1) * 4)) ||
      (st = up(m->inc_tri, inc.data(), 3 * (size_t)t_c * 4)))
    return cleanup_fail(st);
  if ((st = launch_assemble_values(m, 0))) return cleanup_fail(st);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cleanup_fail(cuda_fail(e, "assemble kernels"));
  *out = m;
  return CGP_OK;
}

extern "C" int cgp_mesh_query(cgp_mesh m, int* n_c, int* t_c, int* n_e, int* n_f, int* t_f, int* nnz) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_mesh_query: NULL mesh");
  if (n_c) *n_c = m->n_c;
  if (t_c) *t_c = m->t_c;
  if (n_e) *n_e = m->n_e;
  if (n_f) *n_f = m->n_f;
  if (t_f) *t_f = m->t_f;
  if (nnz) *nnz = m->nnz;
  return CGP_OK;
}

// Nodes of the outer boundary: boundary edges (sides of exactly one triangle)
// oriented as in their counter-clockwise triangle form closed loops; a loop
// around the domain runs counter-clockwise (positive signed area), a loop
// around a hole clockwise.
static std::vector<int> outer_boundary_nodes(const cgp_mesh_impl* m, const double* xy) {
  const int n = m->n_c, t = m->t_c;
  std::vector<std::pair<long long, int>> sides(3 * (size_t)t);   // (undirected key, directed side)
  for (int q = 0; q < t; ++q)
    for (int k = 0; k < 3; ++k) {
      const int a = m->h_tri_c[3 * q + k], b = m->h_tri_c[3 * q + (k + 1) % 3];
      sides[3 * (size_t)q + k] = {(long long)std::min(a, b) * n + std::max(a, b), 3 * q + k};
    }
  std::sort(sides.begin(), sides.end());
  std::vector<int> next(n, -1);
  for (size_t i = 0; i < sides.size();) {
    size_t j = i;
    while (j < sides.size() && sides[j].first == sides[i].first) ++j;
    if (j - i == 1) {
      const int s = sides[i].second, q = s / 3, k = s % 3;
      next[m->h_tri_c[3 * q + k]] = m->h_tri_c[3 * q + (k + 1) % 3];
    }
    i = j;
  }
  std::vector<int> out;
  std::vector<char> seen(n, 0);
  for (int s = 0; s < n; ++s) {
    if (next[s] < 0 || seen[s]) continue;
    std::vector<int> loop;
    double area2 = 0.0;
    for (int a = s; !seen[a] && next[a] >= 0; a = next[a]) {
      seen[a] = 1;
      loop.push_back(a);
      const int b = next[a];
      area2 += xy[2 * a] * xy[2 * b + 1] - xy[2 * b] * xy[2 * a + 1];
    }
    if (area2 > 0.0) out.insert(out.end(), loop.begin(), loop.end());
  }
  std::sort(out.begin(), out.end());
  return out;
}

extern "C" int cgp_set_far_field(cgp_mesh m, int dirichlet) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_set_far_field: NULL mesh");
  if (dirichlet != 0 && dirichlet != 1) return fail(CGP_ERR_INVALID_ARG, "cgp_set_far_field: dirichlet must be 0 or 1");
  if (dirichlet && !m->dir_base) {
    const size_t n = m->n_c, nz = m->nnz;
    std::vector<double> K(nz), xy(2 * n);
    CGP_CUDA(cudaDeviceSynchronize());
    CGP_CUDA(cudaMemcpy(K.data(), m->K, nz * 8, cudaMemcpyDeviceToHost));
    CGP_CUDA(cudaMemcpy(xy.data(), m->xy_c, 2 * n * 8, cudaMemcpyDeviceToHost));
    m->h_outer = outer_boundary_nodes(m, xy.data());
    if (m->h_outer.empty()) return fail(CGP_ERR_INVALID_ARG, "cgp_set_far_field: the mesh has no outer boundary");
    std::vector<unsigned char> fix(n, 0);
    for (int i : m->h_outer) fix[i] = 1;
    std::vector<float> K32(nz), di32(n);
    std::vector<double> di(n);
    for (size_t i = 0; i < n; ++i) {
      double diag = 0.0;
      for (int k = m->h_rowptr[i]; k < m->h_rowptr[i + 1]; ++k) {
        const int j = m->h_col[k];
        if (j == (int)i) {
          if (fix[i]) K[k] = 1.0;       // identity row of a fixed node
          diag = K[k];
        } else if (fix[i] || fix[j]) {
          K[k] = 0.0;                   // eliminated coupling (the fixed value is zero)
        }
        K32[k] = (float)K[k];
      }
      di[i] = 1.0 / diag;
      di32[i] = (float)di[i];
    }
    const size_t o_k32 = align_up(nz * 8, 256), o_d = o_k32 + align_up(nz * 4, 256),
                 o_d32 = o_d + align_up(n * 8, 256), o_f = o_d32 + align_up(n * 4, 256), bytes = o_f + n;
    void* base = nullptr;
    CGP_CUDA(cudaMalloc(&base, bytes));
    char* b = static_cast<char*>(base);
    cudaError_t e = cudaMemcpy(b, K.data(), nz * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_k32, K32.data(), nz * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_d, di.data(), n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_d32, di32.data(), n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_f, fix.data(), n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(base);
      return cuda_fail(e, "cudaMemcpy(far-field system)");
    }
    m->dir_base = base;
    m->Kd = reinterpret_cast<double*>(b);
    m->Kd32 = reinterpret_cast<float*>(b + o_k32);
    m->dinvd = reinterpret_cast<double*>(b + o_d);
    m->dinvd32 = reinterpret_cast<float*>(b + o_d32);
    m->fixed = reinterpret_cast<unsigned char*>(b + o_f);
  }
  m->far_dirichlet = dirichlet;
  return CGP_OK;
}

extern "C" int cgp_far_field_nodes(cgp_mesh m, int* count, int* nodes) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_far_field_nodes: NULL mesh");
  if (!m->dir_base) return fail(CGP_ERR_INVALID_ARG, "cgp_far_field_nodes: call cgp_set_far_field(m, 1) first");
  if (count) *count = (int)m->h_outer.size();
  if (nodes) std::memcpy(nodes, m->h_outer.data(), m->h_outer.size() * 4);
  return CGP_OK;
}

extern "C" int cgp_mesh_levels(cgp_mesh m, int* levels, int* nodes) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_mesh_levels: NULL mesh");
  if (levels) *levels = m->levels;
  if (nodes) std::memcpy(nodes, m->h_lvl_nodes.data(), m->h_lvl_nodes.size() * 4);
  return CGP_OK;
}

extern "C" int cgp_mesh_fine_geometry(cgp_mesh m, double* xy_f, int* tri_f, int* edges) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_mesh_fine_geometry: NULL mesh");
  if (xy_f) CGP_CUDA(cudaMemcpy(xy_f, m->xy_f, 2 * (size_t)m->n_f * 8, cudaMemcpyDeviceToHost));
  if (edges) std::memcpy(edges, m->h_edges.data(), 2 * (size_t)m->n_e * 4);
  if (tri_f) {
    const std::vector<int>& tp = m->levels >= 2 ? m->h_tri_par : m->h_tri_c;
    const std::vector<int>& mp = m->levels >= 2 ? m->h_mid_par : m->h_tri_mid;
    for (int t = 0; t < m->t_par; ++t) {
      const int a = tp[3 * t], b = tp[3 * t + 1], c = tp[3 * t + 2];
      const int mab = mp[3 * t], mbc = mp[3 * t + 1], mca = mp[3 * t + 2];
      const int ch[4][3] = {{a, mab, mca}, {mab, b, mbc}, {mca, mbc, c}, {mab, mbc, mca}};
      for (int k = 0; k < 4; ++k)
        for (int l = 0; l < 3; ++l) tri_f[(size_t)(4 * t + k) * 3 + l] = ch[k][l];
    }
  }
  return CGP_OK;
}

extern "C" int cgp_mesh_matrices(cgp_mesh m, int* rowptr, int* col, double* K, double* Gx, double* Gy,
                                 double* dinv) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_mesh_matrices: NULL mesh");
  const size_t nz = m->nnz;
  if (rowptr) std::memcpy(rowptr, m->h_rowptr.data(), (m->n_c + 1) * 4);
  if (col) std::memcpy(col, m->h_col.data(), nz * 4);
  if (K) CGP_CUDA(cudaMemcpy(K, m->K, nz * 8, cudaMemcpyDeviceToHost));
  if (Gx) CGP_CUDA(cudaMemcpy(Gx, m->Gx, nz * 8, cudaMemcpyDeviceToHost));
  if (Gy) CGP_CUDA(cudaMemcpy(Gy, m->Gy, nz * 8, cudaMemcpyDeviceToHost));
  if (dinv) CGP_CUDA(cudaMemcpy(dinv, m->dinv, (size_t)m->n_c * 8, cudaMemcpyDeviceToHost));
  return CGP_OK;
}

extern "C" int cgp_mesh_destroy(cgp_mesh m) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_mesh_destroy: NULL mesh");
  cudaDeviceSynchronize();
  for (auto& pl : m->plans)
    if (pl.base) cudaFree(pl.base);
  if (m->vinc_base) cudaFree(m->vinc_base);
  if (m->dir_base) cudaFree(m->dir_base);
  for (auto& ps : m->psys) {
    if (ps.base) cudaFree(ps.base);
    if (ps.plan.base) cudaFree(ps.plan.base);
    if (ps.st_base) cudaFree(ps.st_base);
  }
  if (m->st_base) cudaFree(m->st_base);
  if (m->d_base) cudaFree(m->d_base);
  if (m->h_res) cudaFreeHost(m->h_res);
  delete m;
  return CGP_OK;
}
