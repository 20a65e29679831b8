// Internal declarations shared by the translation units of libcgp.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cgp.h"

namespace cgp {

// thread-local error message; returns the status so callers can `return fail(...)`
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define CGP_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return ::cgp::cuda_fail(e_, #call); \
  } while (0)

// Result record of one solve, written by the persistent kernel.
struct SolveResult {
  int iterations;
  int sweeps;
  int status;
  int timeout;       // set by a block whose barrier gave up
  double rel_rec;
  double rel_true;
  double bnorm;
  unsigned long long t_end;  // device clock (ns) when the solve finished
};

// Tuning of the persistent solver launch (chosen by the autotuner or defaults).
struct SolverTuning {
  int block;          // threads per block (0 = default)
  int lanes;          // lanes per CSR row in the SpMV phases (1, 2, 4, 8, 32; 0 = default)
  int blocks;         // blocks of the persistent grid (0 = chosen from the size)
  int flags;          // bit 0: keep rows in global memory (no shared-memory residency)
};

// Shape of the last persistent launch on a mesh (for reports and tests).
struct PlanRecord {
  int blocks;
  int block;
  int resident;
  int smem;
};

// Row partition of the coarse system over `nblk` solver blocks (contiguous
// chunks of ceil(n / nblk) rows) with, per block, the list of columns it
// reads from rows owned by other blocks.  lcol holds, in CSR order, each
// entry's column renumbered into the block's local index space: own rows
// first (j - r0), then the block's halo columns in ascending order.
struct HaloPlan {
  int nblk = 0;
  int max_rows = 0;
  int max_nnz = 0;
  int max_halo = 0;
  int* lcol = nullptr;   // [nnz]
  int* hptr = nullptr;   // [nblk + 1]
  int* hidx = nullptr;   // [total halo]
  void* base = nullptr;  // the one allocation holding the three arrays
};

// A solve's system with its rows renumbered so that every block's contiguous
// chunk is a compact patch of the mesh (recursive coordinate bisection),
// which shrinks the halo each block rebuilds every iteration.
struct PermSystem {
  int nblk = 0, dirichlet = 0, n = 0;
  std::vector<int> h_rowptr, h_col;   // permuted pattern (host)
  int* perm = nullptr;                // [n] new row -> mesh node
  int* rowptr = nullptr;
  int* col = nullptr;
  double* K = nullptr;
  float* K32 = nullptr;
  double* dinv = nullptr;
  float* dinv32 = nullptr;
  unsigned char* fixed = nullptr;     // Dirichlet rows (permuted), or NULL
  double* bbuf = nullptr;             // [n] b in the new order
  double* xbuf = nullptr;             // [n] x in the new order
  HaloPlan plan;                      // halo lists of the permuted pattern
  void* base = nullptr;
  // O-grid tiles (tiles != 0): blocks own near-rectangles of the (angle, ring)
  // index grid and the product uses the seven-point stencil on a padded box
  int tiles = 0;
  int box_cap = 0;                    // largest box (doubles)
  int st_max_halo = 0;
  double* planes = nullptr;           // [7][n] stencil coefficients in the new order
  int* bpos = nullptr;                // [n] box position of every row in its block's box
  int* bdim = nullptr;                // [nblk] box row length
  int* st_hptr = nullptr;             // [nblk + 1] halo of every box (rows read from other blocks)
  int* st_hidx = nullptr;             // [total] their global (new) row
  int* st_hpos = nullptr;             // [total] their box position
  void* st_base = nullptr;
};

struct cgp_mesh_impl {
  int device = 0;
  int n_c = 0, t_c = 0, n_e = 0, n_f = 0, t_f = 0, nnz = 0;
  int levels = 1;                      // 4-way splits between the coarse and the fine mesh (Eq. 18)
  std::vector<int> h_lvl_nodes;        // [levels + 1] nodes of level 0 (coarse) .. levels (fine)
  std::vector<int> h_lvl_eoff;         // [levels + 1] offsets of each level's edges in `edges`
  int t_par = 0;                       // triangles of level levels - 1 (the fine triangles' parents)
  std::vector<int> h_tri_par, h_mid_par;  // levels >= 2: their vertices and edge midpoints (else tri_c, tri_mid)

  // host copies of the integer structure
  std::vector<int> h_rowptr, h_col, h_tri_c, h_edges, h_tri_mid;

  // one device allocation carved into the arrays below
  void* d_base = nullptr;
  size_t d_bytes = 0;

  int* rowptr = nullptr;     // [n_c + 1]
  int* col = nullptr;        // [nnz]
  double* K = nullptr;       // [nnz]
  double* Gx = nullptr;      // [nnz]
  double* Gy = nullptr;      // [nnz]
  double* dinv = nullptr;    // [n_c]
  float* K32 = nullptr;      // [nnz]
  float* dinv32 = nullptr;   // [n_c]
  int* tri_c = nullptr;      // [t_c * 3]
  int* tri_mid = nullptr;    // [t_c * 3]: fine indices of m_ab, m_bc, m_ca
  int* edges = nullptr;      // [2 * all levels' edges]: level 0 (the coarse edges, n_e of them) first
  int* tri_par = nullptr;    // [3 t_par] parents of the fine triangles (tri_c when levels == 1)
  int* mid_par = nullptr;    // [3 t_par] their midpoints m_ab, m_bc, m_ca (tri_mid when levels == 1)
  double* xy_f = nullptr;    // [n_f * 2] interleaved
  double* xy_c = nullptr;    // [n_c * 2]
  int* inc_ptr = nullptr;    // [n_c + 1] node -> incident triangles
  int* inc_tri = nullptr;    // [3 t_c] triangle * 4 + local vertex

  // solver scratch
  double* bp = nullptr;      // projected b
  double* r = nullptr;
  double* z = nullptr;
  double* p = nullptr;
  double* p2 = nullptr;
  double* q = nullptr;
  double* pub64 = nullptr;   // [18 n] published vectors: single-reduction R[2], W[2], S[2] (6 n doubles);
                             // pipelined tagged W[3], Z[3], N[3] (9 n 16-byte words)
  float* f32pub = nullptr;   // [6 n] mixed: published R[2], W[2], S[2]
  float* f32own = nullptr;   // [6 n] mixed without shared-memory residency: own inner vectors
  float* fpart = nullptr;    // [8 * max_blocks] FP32 partial sums
  double* part = nullptr;    // [max_blocks * 32] per-block fixed-point partial sums
  unsigned long long* tpart = nullptr;  // [2][3][max_blocks] tagged 128-bit partial sums
  unsigned* nflag = nullptr; // [max_blocks] pipelined tiles: published-w counts of the blocks
  unsigned* bar = nullptr;   // grid barrier counter
  SolveResult* res = nullptr;
  SolveResult* h_res = nullptr;  // pinned host mirror
  int max_blocks = 0;

  // seven-plane stencil form of K for an O-grid (cgp_mesh_set_ogrid)
  int st_nt = 0, st_nj = 0;
  double* st_val = nullptr;   // [7][n_c]
  float* st_val32 = nullptr;  // [7][n_c]
  void* st_base = nullptr;

  // far-field Dirichlet variant (phi = 0 on the outer boundary), built on first use
  int far_dirichlet = 0;
  std::vector<int> h_outer;        // coarse nodes on the outer boundary loops
  unsigned char* fixed = nullptr;  // [n_c] 1 on those nodes
  double* Kd = nullptr;            // [nnz] K with their rows and columns replaced by the identity
  float* Kd32 = nullptr;
  double* dinvd = nullptr;         // [n_c]
  float* dinvd32 = nullptr;
  void* dir_base = nullptr;

  // fine node -> incident fine triangles, each entry the other two vertices in
  // counter-clockwise order (built on the first velocity correction)
  int* vinc_ptr = nullptr;   // [n_f + 1]
  int* vinc = nullptr;       // [3 t_f][2]
  void* vinc_base = nullptr;

  std::vector<HaloPlan> plans;   // cached per block count
  std::vector<PermSystem> psys;  // cached per (block count, boundary condition, tiles)
  SolverTuning tune[4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};  // by cgp_tune_target
  PlanRecord last_plan[2] = {{0, 0, 0, 0}, {0, 0, 0, 0}};                          // FP64, MIXED
};

// ---- launchers implemented in the .cu files ----
int launch_assemble_values(cgp_mesh_impl* m, cudaStream_t s);
int launch_restrict_rhs(cgp_mesh_impl* m, int kind, double bz, double rho_over_dt,
                        const double* u_f, const double* v_f, double* u_c, double* v_c,
                        double* b, cudaStream_t s);
int launch_prolong(cgp_mesh_impl* m, const double* xc, double* xf, cudaStream_t s);
int launch_velocity_correct(cgp_mesh_impl* m, const double* p_f, const double* u_t, const double* v_t,
                            double dt_over_rho, double* u, double* v, cudaStream_t s);
int launch_lorentz(cgp_mesh_impl* m, const double* phi, const double* u, const double* v,
                   const double B[3], double sigma, double* grad, double* force, cudaStream_t s);
int launch_spmv(cgp_mesh_impl* m, int precision, const void* x, void* y, cudaStream_t s);
int launch_spmv_stencil(cgp_mesh_impl* m, int precision, const void* x, void* y, int block, cudaStream_t s);
int launch_solve(cgp_mesh_impl* m, const double* b, double* x, const cgp_solve_opts& o,
                 cgp_solve_info* info_dev, cudaStream_t s);
int solver_max_blocks(int device);

// FP64 solve of a caller-described CSR system with caller-provided scratch
// (the same persistent kernel as launch_solve, default launch shape).
struct RawSystem {
  int n;
  const int* rowptr;
  const int* col;
  const double* val;
  const double* dinv;
};
struct RawScratch {
  double* bp;
  double* r;
  double* z;
  double* p;
  double* p2;
  double* q;
  double* part;     // [32 * max_blocks]
  int max_blocks;
  unsigned* bar;    // zeroed by the caller before the launch
  SolveResult* res; // zeroed by the caller before the launch
};
int launch_solve_fp64_raw(int device, const RawSystem& sys, const RawScratch& scr, const double* b, double* x,
                          const cgp_solve_opts& o, cudaStream_t s);

}  // namespace cgp

struct cgp_mesh_s : public cgp::cgp_mesh_impl {};
