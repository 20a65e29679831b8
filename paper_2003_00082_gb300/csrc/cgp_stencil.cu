// Structured stencil form of the coarse stiffness matrix of an O-grid.
//
// On the n_theta x n_r O-grid (node (j, i) = j * n_theta + i, ring j from the
// cylinder outwards, angle i periodic, every quad cut along its (i, j) -
// (i+1, j+1) diagonal) every row of K has at most seven entries at fixed
// offsets: (0,0), (+-1,0), (0,+-1), (+1,+1), (-1,-1) in (angle, ring).
// Storing K as seven planes of values indexed by row, with zeros where a
// neighbour does not exist (first and last ring), drops the column indices
// and the row pointers: a product moves 9 s n bytes instead of about
// 12 s n + 4 n (s the value size), the "structured-stencil" alternative to
// CSR for the paper's O-grid-like meshes.
#include <algorithm>
#include <cstring>
#include <vector>

#include "cgp_internal.h"

namespace cgp {
namespace {

constexpr int NS = 7;
// (angle, ring) offset of stencil entry k
__host__ __device__ constexpr int st_di(int k) { return k == 1 || k == 5 ? 1 : (k == 2 || k == 6 ? -1 : 0); }
__host__ __device__ constexpr int st_dj(int k) { return k == 3 || k == 5 ? 1 : (k == 4 || k == 6 ? -1 : 0); }

// y = K x, one row per thread; rows of one ring are consecutive, so the plane
// reads and most x reads are coalesced.
template <typename V>
__global__ void __launch_bounds__(256) stencil_spmv_kernel(int nt, int nj, const V* __restrict__ planes,
                                                           const V* __restrict__ x, V* __restrict__ y) {
  const int n = nt * nj;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int j = row / nt, i = row - j * nt;
  V s = V(0);
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int jj = min(max(j + st_dj(k), 0), nj - 1);   // missing neighbours carry a zero value
    int ii = i + st_di(k);
    ii = ii < 0 ? ii + nt : (ii >= nt ? ii - nt : ii);
    s = fma(planes[(size_t)k * n + row], __ldg(x + (size_t)jj * nt + ii), s);
  }
  y[row] = s;
}

}  // namespace

int launch_spmv_stencil(cgp_mesh_impl* m, int precision, const void* x, void* y, int block, cudaStream_t s) {
  if (!m->st_base) return fail(CGP_ERR_INVALID_ARG, "cgp_spmv: the stencil form needs cgp_mesh_set_ogrid first");
  const int n = m->n_c, bs = block > 0 ? block : 256;
  if (precision == CGP_FP64)
    stencil_spmv_kernel<double><<<(n + bs - 1) / bs, bs, 0, s>>>(m->st_nt, m->st_nj, m->st_val,
                                                                 (const double*)x, (double*)y);
  else
    stencil_spmv_kernel<float><<<(n + bs - 1) / bs, bs, 0, s>>>(m->st_nt, m->st_nj, m->st_val32,
                                                                (const float*)x, (float*)y);
  CGP_CUDA(cudaGetLastError());
  return CGP_OK;
}

}  // namespace cgp

using namespace cgp;

extern "C" int cgp_mesh_set_ogrid(cgp_mesh m, int n_theta, int n_r) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_mesh_set_ogrid: NULL mesh");
  if (n_theta < 3 || n_r < 1 || (long long)n_theta * (n_r + 1) != m->n_c)
    return fail(CGP_ERR_INVALID_ARG, "cgp_mesh_set_ogrid: n_theta * (n_r + 1) must equal n_c, n_theta >= 3, n_r >= 1");
  const int nt = n_theta, nj = n_r + 1, n = m->n_c;
  std::vector<double> K(m->nnz);
  CGP_CUDA(cudaDeviceSynchronize());
  CGP_CUDA(cudaMemcpy(K.data(), m->K, (size_t)m->nnz * 8, cudaMemcpyDeviceToHost));
  std::vector<double> planes((size_t)NS * n, 0.0);
  for (int row = 0; row < n; ++row) {
    const int j = row / nt, i = row % nt;
    int expected = 0;
    for (int k = 0; k < NS; ++k) {
      const int jj = j + st_dj(k);
      if (jj < 0 || jj >= nj) continue;
      ++expected;
      const int ii = (i + st_di(k) + nt) % nt, col = jj * nt + ii;
      const int* b = m->h_col.data() + m->h_rowptr[row];
      const int* e = m->h_col.data() + m->h_rowptr[row + 1];
      const int* f = std::lower_bound(b, e, col);
      if (f == e || *f != col)
        return fail(CGP_ERR_INVALID_ARG, "cgp_mesh_set_ogrid: row " + std::to_string(row) +
                                             " does not have the O-grid stencil (missing column)");
      planes[(size_t)k * n + row] = K[m->h_rowptr[row] + (f - b)];
    }
    if (m->h_rowptr[row + 1] - m->h_rowptr[row] != expected)
      return fail(CGP_ERR_INVALID_ARG, "cgp_mesh_set_ogrid: row " + std::to_string(row) +
                                           " has entries outside the O-grid stencil");
  }
  std::vector<float> p32(planes.size());
  for (size_t q = 0; q < planes.size(); ++q) p32[q] = (float)planes[q];
  if (m->st_base) {
    cudaFree(m->st_base);
    m->st_base = nullptr;
  }
  const size_t b64 = planes.size() * 8, o32 = (b64 + 255) / 256 * 256;
  void* base = nullptr;
  CGP_CUDA(cudaMalloc(&base, o32 + planes.size() * 4));
  cudaError_t e = cudaMemcpy(base, planes.data(), b64, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(static_cast<char*>(base) + o32, p32.data(), p32.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(base);
    return cuda_fail(e, "cudaMemcpy(stencil planes)");
  }
  m->st_base = base;
  m->st_val = static_cast<double*>(base);
  m->st_val32 = reinterpret_cast<float*>(static_cast<char*>(base) + o32);
  m->st_nt = nt;
  m->st_nj = nj;
  return CGP_OK;
}
