// FP64 Poisson solve that allocates nothing.
//
// Some callers cannot call cudaMalloc at solve time: code running under a
// memory pool or arena it does not own, an embedding host whose allocator
// must not be bypassed, or a real-time loop where an allocation (and the
// device synchronisation it can imply) is not allowed.  This entry point
// serves them: the caller passes the CSR system, b and x, and the solver's
// scratch (residual, search direction, partial sums, barrier counter and
// result record) comes from one file-scope device array that every GPU
// loading this library holds until the process exits.
//
// The array is sized for systems of up to CGP_STATIC_MAX_ROWS rows.  All
// calls share it and it keeps the previous call's contents, so the entry
// point clears the barrier counter and the result record before each
// launch; two calls that overlap on the GPU (on different streams, or from
// different host threads) race on it and must be serialised by the caller.
#include <cuda.h>

#include <cstring>
#include <mutex>
#include <string>

#include "cgp_internal.h"

namespace {

constexpr int kStaticMaxRows = 1 << 16;   // matches CGP_STATIC_MAX_ROWS in cgp.h
constexpr int kStaticMaxBlocks = 1024;

// byte layout of the scratch array (every piece 256-byte aligned)
constexpr size_t kVec = (size_t)kStaticMaxRows * sizeof(double);
constexpr size_t kOffBp = 0;
constexpr size_t kOffR = kOffBp + kVec;
constexpr size_t kOffZ = kOffR + kVec;
constexpr size_t kOffP = kOffZ + kVec;
constexpr size_t kOffP2 = kOffP + kVec;
constexpr size_t kOffQ = kOffP2 + kVec;
constexpr size_t kOffPart = kOffQ + kVec;
constexpr size_t kOffBar = kOffPart + (size_t)32 * kStaticMaxBlocks * sizeof(double);
constexpr size_t kOffRes = kOffBar + 256;
constexpr size_t kStaticBytes = kOffRes + 256;
static_assert(sizeof(cgp::SolveResult) <= 256, "result record must fit its slot");

static __device__ __align__(256) unsigned char g_cgp_static_scratch[kStaticBytes];

std::mutex g_mu;

// The array's device address belongs to the CUDA context it was looked up
// in.  Each device's entry keeps the identity of that context (cuCtxGetId,
// unique for the life of the process), so after the caller resets the
// device (cudaDeviceReset, or a reset of the primary context) the next call
// looks the address up again instead of using a stale one.
struct ScratchAddr {
  unsigned long long ctx_id = 0;   // 0: no valid entry
  void* addr = nullptr;
};
ScratchAddr g_addr[256];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Identity of the context current on this thread, or 0 when none is current
// or the driver cannot tell (then every call looks the address up again).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {   // called with g_mu held
    resolved = true;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void**>(&get_current), 12000,
                                         cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess)
      get_current = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void**>(&get_id), 12000,
                                         cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess)
      get_id = nullptr;
    cudaGetLastError();
  }
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current device's context (the
// host-side name of the array is not a device address).  Looked up once per
// device and context, with that device current.
int scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= 256) return cgp::fail(CGP_ERR_INVALID_ARG, "cgp_poisson_solve_noalloc: device id");
  std::lock_guard<std::mutex> lk(g_mu);
  ScratchAddr& a = g_addr[device];
  const unsigned long long id = current_context_id();
  if (id == 0 || a.ctx_id != id || !a.addr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_cgp_static_scratch);
    if (e != cudaSuccess) return cgp::cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    a.addr = p;
    a.ctx_id = current_context_id();   // the lookup has made the device's context current
  }
  *out = static_cast<unsigned char*>(a.addr);
  return CGP_OK;
}

}  // namespace

using namespace cgp;

extern "C" int cgp_poisson_solve_noalloc(int n, const int* rowptr, const int* col, const double* K,
                                         const double* dinv, const double* b, double* x,
                                         const cgp_solve_opts* opts, cgp_solve_info* info, void* stream) {
  if (n < 1 || n > kStaticMaxRows)
    return fail(CGP_ERR_INVALID_ARG, "cgp_poisson_solve_noalloc: n = " + std::to_string(n) +
                                         " is outside [1, " + std::to_string(kStaticMaxRows) +
                                         "], the size of the library's static scratch");
  if (!rowptr || !col || !K || !dinv || !b || !x)
    return fail(CGP_ERR_INVALID_ARG, "cgp_poisson_solve_noalloc: NULL pointer argument");
  cgp_solve_opts o{1e-8, 20000, CGP_FP64, 1e-4, 0, 50};
  if (opts) o = *opts;
  if (o.precision != CGP_FP64) return fail(CGP_ERR_INVALID_ARG, "cgp_poisson_solve_noalloc: FP64 only");
  if (!(o.tol >= 0.0) || o.max_it < 0) return fail(CGP_ERR_INVALID_ARG, "cgp_poisson_solve_noalloc: bad tol or max_it");

  int device = 0;
  CGP_CUDA(cudaGetDevice(&device));
  unsigned char* base = nullptr;
  int st = scratch_address(device, &base);
  if (st != CGP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;

  RawScratch scr{};
  scr.bp = reinterpret_cast<double*>(base + kOffBp);
  scr.r = reinterpret_cast<double*>(base + kOffR);
  scr.z = reinterpret_cast<double*>(base + kOffZ);
  scr.p = reinterpret_cast<double*>(base + kOffP);
  scr.p2 = reinterpret_cast<double*>(base + kOffP2);
  scr.q = reinterpret_cast<double*>(base + kOffQ);
  scr.part = reinterpret_cast<double*>(base + kOffPart);
  scr.max_blocks = kStaticMaxBlocks;
  scr.bar = reinterpret_cast<unsigned*>(base + kOffBar);
  scr.res = reinterpret_cast<SolveResult*>(base + kOffRes);
  // the array keeps the last call's contents: restart the barrier and the record
  CGP_CUDA(cudaMemsetAsync(base + kOffBar, 0, 512, s));

  RawSystem sys{n, rowptr, col, K, dinv};
  st = launch_solve_fp64_raw(device, sys, scr, b, x, o, s);
  if (st != CGP_OK || !info) return st;

  SolveResult r;
  std::memset(&r, 0, sizeof(r));
  CGP_CUDA(cudaMemcpyAsync(&r, scr.res, sizeof(SolveResult), cudaMemcpyDeviceToHost, s));
  CGP_CUDA(cudaStreamSynchronize(s));
  info->iterations = r.iterations;
  info->outer_sweeps = 0;
  info->rel_res_recursive = r.rel_rec;
  info->rel_res_true = r.rel_true;
  info->status = r.timeout ? CGP_ERR_TIMEOUT : r.status;
  if (info->status != CGP_OK) return fail(info->status, "cgp_poisson_solve_noalloc: solve did not succeed");
  return CGP_OK;
}
