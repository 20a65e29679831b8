// Mapping operators and the fine-mesh outputs of a CGP step.
//
//   restrict_rhs : injection u_c = u_f[0, n_c) (Eq. 19) fused with the weak
//                  Poisson right-hand side b = Gx F_x + Gy F_y (Eqs. 12, 15).
//   prolong      : Eq. 20 on the 4-way split: coarse nodes copy, edge
//                  midpoints average their two end values.
//   lorentz      : per fine triangle grad(phi), j = sigma(-grad phi + u x B)
//                  (Eqs. 4, 7) and f = j x B (Eqs. 2, 8, 13-14), one thread per
//                  coarse triangle producing its four children.
#include "cgp_internal.h"

namespace cgp {
namespace {

// One thread per coarse row.  F is formed from the fine velocity at the
// coarse nodes (the prefix of the fine numbering), so no restricted copy is
// needed; it is written only when the caller asks for it.
template <int KIND>
__global__ void restrict_rhs_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                    const double* __restrict__ Gx, const double* __restrict__ Gy,
                                    double bz, double rho_over_dt, const double* __restrict__ u_f,
                                    const double* __restrict__ v_f, double* __restrict__ u_c,
                                    double* __restrict__ v_c, double* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sx = 0.0, sy = 0.0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const int j = col[k];
    const double u = u_f[j], v = v_f[j];
    double fx, fy;
    if (KIND == CGP_RHS_POTENTIAL) {  // in-plane part of u x B with u_z = 0
      fx = v * bz;
      fy = -(u * bz);
    } else {                           // (rho / dt) u~
      fx = rho_over_dt * u;
      fy = rho_over_dt * v;
    }
    sx = fma(Gx[k], fx, sx);
    sy = fma(Gy[k], fy, sy);
  }
  b[i] = sx + sy;
  if (u_c) u_c[i] = u_f[i];
  if (v_c) v_c[i] = v_f[i];
}

// Two fine nodes per thread: coarse prefix copy, then midpoints.
__global__ void prolong_kernel(int n_c, int n_f, const int2* __restrict__ edges,
                               const double* __restrict__ xc, double* __restrict__ xf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_f) return;
  if (i < n_c) {
    xf[i] = xc[i];
  } else {
    const int2 e = edges[i - n_c];
    xf[i] = (xc[e.x] + xc[e.y]) * 0.5;
  }
}

struct Node {
  double x, y, phi, u, v;
};

__device__ __forceinline__ Node load_node(int i, const double2* __restrict__ xy,
                                          const double* __restrict__ phi,
                                          const double* __restrict__ u,
                                          const double* __restrict__ v) {
  const double2 p = xy[i];
  return Node{p.x, p.y, phi[i], u[i], v[i]};
}

// grad(phi) on the P1 triangle (n0, n1, n2), then Ohm's law and j x B.
__device__ __forceinline__ void child(const Node& n0, const Node& n1, const Node& n2, double bx,
                                      double by, double bz, double sigma, double& gx, double& gy,
                                      double& fx, double& fy) {
  const double b0 = n1.y - n2.y, b1 = n2.y - n0.y, b2 = n0.y - n1.y;
  const double c0 = n2.x - n1.x, c1 = n0.x - n2.x, c2 = n1.x - n0.x;
  const double a2 = (n1.x - n0.x) * (n2.y - n0.y) - (n2.x - n0.x) * (n1.y - n0.y);
  const double inv = 1.0 / a2;
  gx = (n0.phi * b0 + n1.phi * b1 + n2.phi * b2) * inv;
  gy = (n0.phi * c0 + n1.phi * c1 + n2.phi * c2) * inv;
  const double ub = (n0.u + n1.u + n2.u) * (1.0 / 3.0);
  const double vb = (n0.v + n1.v + n2.v) * (1.0 / 3.0);
  // u x B with u_z = 0
  const double cx = vb * bz, cy = -(ub * bz), cz = ub * by - vb * bx;
  const double jx = sigma * (cx - gx), jy = sigma * (cy - gy), jz = sigma * cz;
  fx = jy * bz - jz * by;
  fy = jz * bx - jx * bz;
}

template <bool FORCE>
__global__ void lorentz_kernel(int t_c, int t_f, const int* __restrict__ tri,
                               const int* __restrict__ mid, const double2* __restrict__ xy,
                               const double* __restrict__ phi, const double* __restrict__ u,
                               const double* __restrict__ v, double bx, double by, double bz,
                               double sigma, double* __restrict__ grad, double* __restrict__ force) {
  const int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= t_c) return;
  const Node a = load_node(tri[3 * T], xy, phi, u, v);
  const Node b = load_node(tri[3 * T + 1], xy, phi, u, v);
  const Node c = load_node(tri[3 * T + 2], xy, phi, u, v);
  const Node mab = load_node(mid[3 * T], xy, phi, u, v);
  const Node mbc = load_node(mid[3 * T + 1], xy, phi, u, v);
  const Node mca = load_node(mid[3 * T + 2], xy, phi, u, v);
  double gx[4], gy[4], fx[4], fy[4];
  child(a, mab, mca, bx, by, bz, sigma, gx[0], gy[0], fx[0], fy[0]);
  child(mab, b, mbc, bx, by, bz, sigma, gx[1], gy[1], fx[1], fy[1]);
  child(mca, mbc, c, bx, by, bz, sigma, gx[2], gy[2], fx[2], fy[2]);
  child(mab, mbc, mca, bx, by, bz, sigma, gx[3], gy[3], fx[3], fy[3]);
  const size_t t0 = 4 * (size_t)T;
  // four consecutive children: 32-byte aligned vector stores
  reinterpret_cast<double4*>(grad + t0)[0] = make_double4(gx[0], gx[1], gx[2], gx[3]);
  reinterpret_cast<double4*>(grad + t_f + t0)[0] = make_double4(gy[0], gy[1], gy[2], gy[3]);
  if (FORCE) {
    reinterpret_cast<double4*>(force + t0)[0] = make_double4(fx[0], fx[1], fx[2], fx[3]);
    reinterpret_cast<double4*>(force + t_f + t0)[0] = make_double4(fy[0], fy[1], fy[2], fy[3]);
  }
}

}  // namespace

int launch_restrict_rhs(cgp_mesh_impl* m, int kind, double bz, double rho_over_dt, const double* u_f,
                        const double* v_f, double* u_c, double* v_c, double* b, cudaStream_t s) {
  const int bs = 256, gs = (m->n_c + bs - 1) / bs;
  if (kind == CGP_RHS_POTENTIAL)
    restrict_rhs_kernel<CGP_RHS_POTENTIAL><<<gs, bs, 0, s>>>(m->n_c, m->rowptr, m->col, m->Gx, m->Gy, bz,
                                                             rho_over_dt, u_f, v_f, u_c, v_c, b);
  else
    restrict_rhs_kernel<CGP_RHS_PRESSURE><<<gs, bs, 0, s>>>(m->n_c, m->rowptr, m->col, m->Gx, m->Gy, bz,
                                                            rho_over_dt, u_f, v_f, u_c, v_c, b);
  CGP_CUDA(cudaGetLastError());
  return CGP_OK;
}

int launch_prolong(cgp_mesh_impl* m, const double* xc, double* xf, cudaStream_t s) {
  const int bs = 256;
  prolong_kernel<<<(m->n_f + bs - 1) / bs, bs, 0, s>>>(m->n_c, m->n_f, reinterpret_cast<const int2*>(m->edges),
                                                       xc, xf);
  CGP_CUDA(cudaGetLastError());
  return CGP_OK;
}

int launch_lorentz(cgp_mesh_impl* m, const double* phi, const double* u, const double* v, const double B[3],
                   double sigma, double* grad, double* force, cudaStream_t s) {
  const int bs = 128, gs = (m->t_c + bs - 1) / bs;
  const double2* xy = reinterpret_cast<const double2*>(m->xy_f);
  if (force)
    lorentz_kernel<true><<<gs, bs, 0, s>>>(m->t_c, m->t_f, m->tri_c, m->tri_mid, xy, phi, u, v, B[0], B[1],
                                           B[2], sigma, grad, force);
  else
    lorentz_kernel<false><<<gs, bs, 0, s>>>(m->t_c, m->t_f, m->tri_c, m->tri_mid, xy, phi, u, v, B[0], B[1],
                                            B[2], sigma, grad, force);
  CGP_CUDA(cudaGetLastError());
  return CGP_OK;
}

}  // namespace cgp

using namespace cgp;

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

extern "C" int cgp_restrict(cgp_mesh m, int kind, const double* B, double rho_over_dt, const double* u_f,
                            const double* v_f, double* u_c, double* v_c, double* b, void* stream) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_restrict: NULL mesh");
  if (!u_f || !v_f || !b) return fail(CGP_ERR_INVALID_ARG, "cgp_restrict: NULL u_f, v_f or b");
  if (kind != CGP_RHS_POTENTIAL && kind != CGP_RHS_PRESSURE)
    return fail(CGP_ERR_INVALID_ARG, "cgp_restrict: unknown kind");
  if (kind == CGP_RHS_POTENTIAL && !B) return fail(CGP_ERR_INVALID_ARG, "cgp_restrict: NULL B");
  const double bz = B ? B[2] : 0.0;
  return launch_restrict_rhs(m, kind, bz, rho_over_dt, u_f, v_f, u_c, v_c, b, (cudaStream_t)stream);
}

extern "C" int cgp_prolong(cgp_mesh m, const double* x_c, double* x_f, void* stream) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_prolong: NULL mesh");
  if (!x_c || !x_f) return fail(CGP_ERR_INVALID_ARG, "cgp_prolong: NULL vector");
  return launch_prolong(m, x_c, x_f, (cudaStream_t)stream);
}

extern "C" int cgp_lorentz(cgp_mesh m, const double* phi_f, const double* u_f, const double* v_f,
                           const double* B, double sigma, double* grad, double* force, void* stream) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_lorentz: NULL mesh");
  if (!phi_f || !grad || !B) return fail(CGP_ERR_INVALID_ARG, "cgp_lorentz: NULL phi_f, grad or B");
  if (force && (!u_f || !v_f)) return fail(CGP_ERR_INVALID_ARG, "cgp_lorentz: force needs u_f and v_f");
  if (!aligned(grad, 32) || (force && !aligned(force, 32)))
    return fail(CGP_ERR_INVALID_ARG, "cgp_lorentz: grad and force must be 32-byte aligned");
  // without force the velocity is not read; pass phi as a valid stand-in pointer
  const double* u = u_f ? u_f : phi_f;
  const double* v = v_f ? v_f : phi_f;
  return launch_lorentz(m, phi_f, u, v, B, sigma, grad, force, (cudaStream_t)stream);
}
