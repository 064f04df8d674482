// Allocation-free fine-level smoothing (ehs_fine_smooth_noalloc in ehs.h).
//
// Who needs this: callers that may not allocate device memory at the point
// where they want to relax a vector, and so cannot build a context (ehs_create
// allocates a whole hierarchy).  Examples: a host program that hands all of
// the device memory to its own pool at start-up and forbids the libraries it
// loads to call cudaMalloc, so that its footprint stays fixed and known; and
// latency-bound loops that must not stall on the allocator (cudaFree waits for
// the whole device).  This entry point keeps its scratch (the matrix-free cell
// coefficients, the per-medium frequencies and the red-black ping-pong vector)
// in one file-scope device array of fixed size that every GPU loading the
// library holds until the process exits, and calls no allocating routine.
//
// The array is shared by every call on a device: calls whose GPU work
// overlaps (different streams, or different host threads) race on it and
// must be serialised by the caller.  The first call on each device looks up
// the array's device address (cudaGetSymbolAddress); make that first call
// before any stream capture begins.
#include <cmath>
#include <mutex>

#include "ehs.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = 32u << 20;   // 32 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDev = 64;
constexpr int kMaxMedia = 32;
void* g_scratch_addr[kMaxDev] = {nullptr};
std::mutex g_scratch_mu;

// the per-medium frequencies, passed to the device by value as a kernel
// argument (no host-to-device copy from host memory that the call owns)
struct Omegas {
  double w[kMaxMedia];
};

__global__ void k_put_omegas(Omegas om, int n, double* dst) {
  const int i = threadIdx.x;
  if (i < n) dst[i] = om.w[i];
}

// the status alone reports the failure (this entry point has no context to
// hold a message); the text documents each case at the call site
inline ehs_status fail(ehs_status st, const char* /*why*/) { return st; }

// device memory of the current device (or managed memory); anything else --
// host memory, or memory of another GPU -- is refused
bool on_this_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

template <typename T>
ehs_status run(const ehs_problem* P, int nrhs, double alpha, double w, double wp, int nsweeps,
               const void* b, void* x, cudaStream_t s, unsigned char* scratch) {
  using namespace ehs;
  typedef typename CT<T>::type C;
  Grid g;
  g.d = P->dim;
  g.n[0] = P->n[0]; g.n[1] = P->n[1]; g.n[2] = P->dim == 3 ? P->n[2] : 1;
  g.ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  const int items = P->nmedia * nrhs;
  const size_t coef_bytes = (size_t)P->nmedia * g.ncell * sizeof(Coef4<T>);
  const size_t vec_bytes = (size_t)items * (g.d + 1) * g.ncell * sizeof(C);
  const size_t om_bytes = 256;
  const size_t cb = (coef_bytes + 255) & ~(size_t)255;
  if (om_bytes + cb + vec_bytes > kScratchBytes)
    return fail(EHS_ERR_OOM, "problem too large for the 32 MiB allocation-free scratch");
  double* d_om = reinterpret_cast<double*>(scratch);
  Coef4<T>* cf = reinterpret_cast<Coef4<T>*>(scratch + om_bytes);
  C* t = reinterpret_cast<C*>(scratch + om_bytes + cb);
  Omegas om{};
  for (int m = 0; m < P->nmedia; ++m) om.w[m] = P->omegas ? P->omegas[m] : P->omega;
  for (int m = 0; m < P->nmedia; ++m)
    if (!std::isfinite(om.w[m]) || !(om.w[m] > 0)) return fail(EHS_ERR_ARG, "omega must be positive and finite");
  // the previous call's contents are still there: the frequencies are
  // overwritten, the coefficients fully rewritten, and the ping-pong vector
  // cleared so that its boundary slots (never written by a sweep) are zero
  k_put_omegas<<<1, kMaxMedia, 0, s>>>(om, P->nmedia, d_om);
  if (cudaMemsetAsync(t, 0, vec_bytes, s) != cudaSuccess)
    return fail(EHS_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  launch_fine_coef<T>(g, P->nmedia, P->lambda, P->mu, P->rho, d_om, P->abl_cells, P->abl_max,
                      P->gamma_add, cf, s);
  for (int k = 0; k < nsweeps; ++k) {
    launch_fine_vanka<T>(g, items, nrhs, cf, P->h, alpha, (T)w, (T)wp, 0, (const C*)b, (const C*)x, t, s);
    launch_fine_vanka<T>(g, items, nrhs, cf, P->h, alpha, (T)w, (T)wp, 1, (const C*)b, t, (C*)x, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(EHS_ERR_CUDA, cudaGetErrorString(e));
  return EHS_OK;
}

}  // namespace

extern "C" ehs_status ehs_fine_smooth_noalloc(const ehs_problem* P, int nrhs, double alpha, double w,
                                              double wp, int nsweeps, int prec, const void* b, void* x,
                                              void* stream) {
  if (!P || !b || !x) return fail(EHS_ERR_ARG, "null argument");
  if (P->dim != 2 && P->dim != 3) return fail(EHS_ERR_ARG, "dim must be 2 or 3");
  int nmin = P->n[0];
  for (int k = 0; k < P->dim; ++k) {
    if (P->n[k] < 2 || P->n[k] % 2) return fail(EHS_ERR_ARG, "every n[k] must be even and >= 2");
    nmin = P->n[k] < nmin ? P->n[k] : nmin;
  }
  if (P->abl_cells < 0 || 2 * P->abl_cells > nmin)
    return fail(EHS_ERR_ARG, "abl_cells must be in [0, min n[k] / 2]");
  if (P->nmedia < 1 || P->nmedia > kMaxMedia || nrhs < 1 || nsweeps < 0)
    return fail(EHS_ERR_ARG, "bad nmedia (1..32), nrhs or nsweeps");
  if (!(P->h > 0)) return fail(EHS_ERR_ARG, "h must be positive");
  if (prec != EHS_C64 && prec != EHS_C128) return fail(EHS_ERR_ARG, "prec must be EHS_C64 or EHS_C128");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
    return fail(EHS_ERR_CUDA, "no current CUDA device");
  if (!P->lambda || !P->mu || !P->rho || !on_this_device(P->lambda, dev) || !on_this_device(P->mu, dev) ||
      !on_this_device(P->rho, dev) || !on_this_device(b, dev) || !on_this_device(x, dev))
    return fail(EHS_ERR_ARG, "media, b and x must be memory of the current device");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return fail(EHS_ERR_CUDA, cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == EHS_C128) return run<double>(P, nrhs, alpha, w, wp, nsweeps, b, x, s, (unsigned char*)scratch);
  return run<float>(P, nrhs, alpha, w, wp, nsweeps, b, x, s, (unsigned char*)scratch);
}
