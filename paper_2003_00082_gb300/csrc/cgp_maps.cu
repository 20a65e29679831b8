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

// One level-1 node per thread: the coarse prefix copied, then the midpoints of the coarse edges.
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

// One further level (Eq. 20 from level l to l + 1, in place): node n_l + e
// is the midpoint of level-l edge e, where the parent's shape functions are
// (1/2, 1/2, 0); level l's nodes are the prefix and already hold their values.
__global__ void prolong_level_kernel(int n_l, int e_l, const int2* __restrict__ edges, double* __restrict__ xf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= e_l) return;
  const int2 ed = edges[e];
  xf[n_l + e] = (xf[ed.x] + xf[ed.y]) * 0.5;
}

// Ohm's law and the force with uniform B, u_z = 0 and the vertex means
// (u_b, v_b) = (su, sv) / 3:  j = sigma (u x B - grad phi) and j x B expand to
//   f_x = -su k1 + sv k2 - g_y k3,   f_y = su k2 - sv k4 + g_x k3,
// k1 = sigma (B_y^2 + B_z^2) / 3, k2 = sigma B_x B_y / 3, k3 = sigma B_z,
// k4 = sigma (B_x^2 + B_z^2) / 3, folded once on the host.
struct ForceCoef {
  double k1, k2, k3, k4;
};

// One fine child of a parent triangle.  A child of the midpoint split is the
// parent scaled by 1/2 (the middle child also turned by half a turn): its
// (b_i, c_i) are the parent's halved (for the middle child negated and
// permuted) and its doubled area is the parent's over 4, so
// grad phi = 2 sum_i phi_i (b_i, c_i) / a2_parent.  One division per parent
// on the GPU's narrow FP64 pipe instead of one per child; the result differs
// from the child's own geometry by rounding only.
template <bool FORCE>
__device__ __forceinline__ void child(double p0, double p1, double p2, double su, double sv, double b0, double b1,
                                      double b2, double c0, double c1, double c2, double inv2, const ForceCoef& k,
                                      double& gx, double& gy, double& fx, double& fy) {
  gx = (p0 * b0 + p1 * b1 + p2 * b2) * inv2;
  gy = (p0 * c0 + p1 * c1 + p2 * c2) * inv2;
  if (FORCE) {
    fx = sv * k.k2 - su * k.k1 - gy * k.k3;
    fy = su * k.k2 - sv * k.k4 + gx * k.k3;
  }
}

template <bool FORCE>
__global__ void lorentz_kernel(int t_c, int t_f, const int* __restrict__ tri,
                               const int* __restrict__ mid, const double2* __restrict__ xy,
                               const double* __restrict__ phi, const double* __restrict__ u,
                               const double* __restrict__ v, ForceCoef k, double* __restrict__ grad,
                               double* __restrict__ force) {
  const int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= t_c) return;
  const int ia = tri[3 * T], ib = tri[3 * T + 1], ic = tri[3 * T + 2];
  const int iab = mid[3 * T], ibc = mid[3 * T + 1], ica = mid[3 * T + 2];
  const double2 xa = xy[ia], xb = xy[ib], xc = xy[ic];
  const double pa = phi[ia], pb = phi[ib], pc = phi[ic], pab = phi[iab], pbc = phi[ibc], pca = phi[ica];
  // vertex sums of u and v for the four children, sharing the midpoint pairs
  double su[4] = {0, 0, 0, 0}, sv[4] = {0, 0, 0, 0};
  if (FORCE) {
    const double uab = u[iab], ubc = u[ibc], uca = u[ica], vab = v[iab], vbc = v[ibc], vca = v[ica];
    const double u_a = uab + uca, u_b = uab + ubc, u_c = uca + ubc;
    const double v_a = vab + vca, v_b = vab + vbc, v_c = vca + vbc;
    su[0] = u[ia] + u_a; su[1] = u[ib] + u_b; su[2] = u[ic] + u_c; su[3] = u_a + ubc;
    sv[0] = v[ia] + v_a; sv[1] = v[ib] + v_b; sv[2] = v[ic] + v_c; sv[3] = v_a + vbc;
  }
  const double b0 = xb.y - xc.y, b1 = xc.y - xa.y, b2 = xa.y - xb.y;
  const double c0 = xc.x - xb.x, c1 = xa.x - xc.x, c2 = xb.x - xa.x;
  const double a2 = (xb.x - xa.x) * (xc.y - xa.y) - (xc.x - xa.x) * (xb.y - xa.y);
  const double inv2 = 2.0 / a2;
  double gx[4], gy[4], fx[4], fy[4];
  child<FORCE>(pa, pab, pca, su[0], sv[0], b0, b1, b2, c0, c1, c2, inv2, k, gx[0], gy[0], fx[0], fy[0]);
  child<FORCE>(pab, pb, pbc, su[1], sv[1], b0, b1, b2, c0, c1, c2, inv2, k, gx[1], gy[1], fx[1], fy[1]);
  child<FORCE>(pca, pbc, pc, su[2], sv[2], b0, b1, b2, c0, c1, c2, inv2, k, gx[2], gy[2], fx[2], fy[2]);
  child<FORCE>(pab, pbc, pca, su[3], sv[3], -b2, -b0, -b1, -c2, -c0, -c1, inv2, k, gx[3], gy[3], fx[3], fy[3]);
  const size_t t0 = 4 * (size_t)T;
  // four consecutive children: 32-byte aligned vector stores
  reinterpret_cast<double4*>(grad + t0)[0] = make_double4(gx[0], gx[1], gx[2], gx[3]);
  reinterpret_cast<double4*>(grad + t_f + t0)[0] = make_double4(gy[0], gy[1], gy[2], gy[3]);
  if (FORCE) {
    reinterpret_cast<double4*>(force + t0)[0] = make_double4(fx[0], fx[1], fx[2], fx[3]);
    reinterpret_cast<double4*>(force + t_f + t0)[0] = make_double4(fy[0], fy[1], fy[2], fy[3]);
  }
}

// Velocity correction (Eqs. 16-17) at fine node i with the lumped P1 mass:
// u_i = u~_i - (dt/rho) sum_T |T| dp/dx|_T / sum_T |T| over the fine
// triangles T around i.  For T = (i, j, k) counter-clockwise,
// 2|T| grad p = (p_i (y_j - y_k) + p_j (y_k - y_i) + p_k (y_i - y_j),
//                p_i (x_k - x_j) + p_j (x_i - x_k) + p_k (x_j - x_i)),
// so the weights 2|T| cancel the division by the area.  Triangles are taken
// in increasing index order (deterministic).
__global__ void velocity_correct_kernel(int n_f, const int* __restrict__ ptr, const int2* __restrict__ inc,
                                        const double2* __restrict__ xy, const double* __restrict__ p,
                                        const double* __restrict__ ut, const double* __restrict__ vt,
                                        double c, double* __restrict__ u, double* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_f) return;
  const double2 xi = xy[i];
  const double pi = p[i];
  double sx = 0.0, sy = 0.0, sa = 0.0;
  for (int q = ptr[i]; q < ptr[i + 1]; ++q) {
    const int2 jk = inc[q];
    const double2 xj = xy[jk.x], xk = xy[jk.y];
    const double pj = p[jk.x], pk = p[jk.y];
    sx += pi * (xj.y - xk.y) + pj * (xk.y - xi.y) + pk * (xi.y - xj.y);
    sy += pi * (xk.x - xj.x) + pj * (xi.x - xk.x) + pk * (xj.x - xi.x);
    sa += (xj.x - xi.x) * (xk.y - xi.y) - (xk.x - xi.x) * (xj.y - xi.y);
  }
  const double ia = 1.0 / sa;
  u[i] = ut[i] - c * (sx * ia);
  v[i] = vt[i] - c * (sy * ia);
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
  const int n1 = m->h_lvl_nodes[1];
  prolong_kernel<<<(n1 + bs - 1) / bs, bs, 0, s>>>(m->n_c, n1, reinterpret_cast<const int2*>(m->edges), xc, xf);
  CGP_CUDA(cudaGetLastError());
  for (int l = 1; l < m->levels; ++l) {   // one launch per further level, as Eq. 20 prolongs one level at a time
    const int e_l = m->h_lvl_eoff[l + 1] - m->h_lvl_eoff[l];
    prolong_level_kernel<<<(e_l + bs - 1) / bs, bs, 0, s>>>(
        m->h_lvl_nodes[l], e_l, reinterpret_cast<const int2*>(m->edges) + m->h_lvl_eoff[l], xf);
    CGP_CUDA(cudaGetLastError());
  }
  return CGP_OK;
}

int launch_lorentz(cgp_mesh_impl* m, const double* phi, const double* u, const double* v, const double B[3],
                   double sigma, double* grad, double* force, cudaStream_t s) {
  // one thread per parent (level levels - 1) triangle and its four fine children
  const int bs = 128, gs = (m->t_par + bs - 1) / bs;
  const double2* xy = reinterpret_cast<const double2*>(m->xy_f);
  const ForceCoef k{sigma * (B[1] * B[1] + B[2] * B[2]) / 3.0, sigma * B[0] * B[1] / 3.0, sigma * B[2],
                    sigma * (B[0] * B[0] + B[2] * B[2]) / 3.0};
  if (force)
    lorentz_kernel<true><<<gs, bs, 0, s>>>(m->t_par, m->t_f, m->tri_par, m->mid_par, xy, phi, u, v, k, grad, force);
  else
    lorentz_kernel<false><<<gs, bs, 0, s>>>(m->t_par, m->t_f, m->tri_par, m->mid_par, xy, phi, u, v, k, grad, force);
  CGP_CUDA(cudaGetLastError());
  return CGP_OK;
}

// Fine-node incidence for the velocity correction, built once per mesh on the host.
static int build_vinc(cgp_mesh_impl* m) {
  if (m->vinc) return CGP_OK;
  const std::vector<int>& tp = m->levels >= 2 ? m->h_tri_par : m->h_tri_c;
  const std::vector<int>& mp = m->levels >= 2 ? m->h_mid_par : m->h_tri_mid;
  const size_t nf = m->n_f, tf = m->t_f;
  std::vector<int> ptr(nf + 1, 0), ent(6 * tf);
  auto fine_tri = [&](size_t t, int (&v)[3]) {
    const size_t T = t / 4;
    const int a = tp[3 * T], b = tp[3 * T + 1], c = tp[3 * T + 2];
    const int mab = mp[3 * T], mbc = mp[3 * T + 1], mca = mp[3 * T + 2];
    const int ch[4][3] = {{a, mab, mca}, {mab, b, mbc}, {mca, mbc, c}, {mab, mbc, mca}};
    for (int l = 0; l < 3; ++l) v[l] = ch[t % 4][l];
  };
  int v[3];
  for (size_t t = 0; t < tf; ++t) {
    fine_tri(t, v);
    for (int l = 0; l < 3; ++l) ptr[v[l] + 1]++;
  }
  for (size_t i = 0; i < nf; ++i) ptr[i + 1] += ptr[i];
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (size_t t = 0; t < tf; ++t) {
    fine_tri(t, v);
    for (int l = 0; l < 3; ++l) {
      const int q = fill[v[l]]++;
      ent[2 * (size_t)q] = v[(l + 1) % 3];
      ent[2 * (size_t)q + 1] = v[(l + 2) % 3];
    }
  }
  const size_t b_ptr = (nf + 1) * 4, o_inc = (b_ptr + 255) / 256 * 256;
  void* base = nullptr;
  CGP_CUDA(cudaMalloc(&base, o_inc + ent.size() * 4));
  cudaError_t e = cudaMemcpy(base, ptr.data(), b_ptr, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(static_cast<char*>(base) + o_inc, ent.data(), ent.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(base);
    return cuda_fail(e, "cudaMemcpy(fine incidence)");
  }
  m->vinc_base = base;
  m->vinc_ptr = static_cast<int*>(base);
  m->vinc = reinterpret_cast<int*>(static_cast<char*>(base) + o_inc);
  return CGP_OK;
}

int launch_velocity_correct(cgp_mesh_impl* m, const double* p_f, const double* u_t, const double* v_t,
                            double dt_over_rho, double* u, double* v, cudaStream_t s) {
  int st = build_vinc(m);
  if (st != CGP_OK) return st;
  const int bs = 256;
  velocity_correct_kernel<<<(m->n_f + bs - 1) / bs, bs, 0, s>>>(
      m->n_f, m->vinc_ptr, reinterpret_cast<const int2*>(m->vinc), reinterpret_cast<const double2*>(m->xy_f), p_f,
      u_t, v_t, dt_over_rho, u, v);
  CGP_CUDA(cudaGetLastError());
  return CGP_OK;
}

}  // namespace cgp

using namespace cgp;

extern "C" int cgp_velocity_correct(cgp_mesh m, const double* p_f, const double* u_t, const double* v_t,
                                    double dt_over_rho, double* u, double* v, void* stream) {
  if (!m) return fail(CGP_ERR_INVALID_ARG, "cgp_velocity_correct: NULL mesh");
  if (!p_f || !u_t || !v_t || !u || !v) return fail(CGP_ERR_INVALID_ARG, "cgp_velocity_correct: NULL vector");
  if (!(dt_over_rho == dt_over_rho)) return fail(CGP_ERR_INVALID_ARG, "cgp_velocity_correct: dt_over_rho is NaN");
  return launch_velocity_correct(m, p_f, u_t, v_t, dt_over_rho, u, v, (cudaStream_t)stream);
}

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
