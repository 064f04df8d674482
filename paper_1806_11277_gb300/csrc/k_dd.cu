// Restriction of the global residual to padded subdomains and scatter-add of
// their corrections (Algorithm DD steps 1 and 3).  Sub-item b_l =
// ((m * nsub) + s) * nrhs + r belongs to medium m, subdomain s, source r and
// reads/writes global item m * nrhs + r.  map[s][e] is the global slot of
// local slot e, or -1 outside Omega_i (padding and its interface faces).
#include "kernels.h"

namespace ehs {
namespace {

template <typename C>
__global__ void k_dd_gather(long long nl, int nsub, int nrhs, long long ng, const int* __restrict__ map,
                            const C* __restrict__ res, C* __restrict__ out, const int* __restrict__ il) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nl) return;
  const int bl = il ? il[blockIdx.y] : blockIdx.y;
  const int r = bl % nrhs, s = (bl / nrhs) % nsub, m = bl / (nrhs * nsub);
  const int gs = map[(long long)s * nl + e];
  C v; v.x = 0; v.y = 0;
  if (gs >= 0) v = res[(long long)(m * nrhs + r) * ng + gs];
  out[(long long)bl * nl + e] = v;
}

template <typename C>
__global__ void k_dd_scatter(long long nl, int nsub, int nrhs, long long ng, const int* __restrict__ map,
                             const C* __restrict__ xs, C* __restrict__ x, const int* __restrict__ il) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nl) return;
  const int bl = il ? il[blockIdx.y] : blockIdx.y;
  const int r = bl % nrhs, s = (bl / nrhs) % nsub, m = bl / (nrhs * nsub);
  const int gs = map[(long long)s * nl + e];
  if (gs < 0) return;
  const C v = xs[(long long)bl * nl + e];
  C& t = x[(long long)(m * nrhs + r) * ng + gs];
  t.x += v.x;
  t.y += v.y;
}

__global__ void k_expand_items(const int* __restrict__ list, int nact, int nrhs, int nsub,
                               const int* __restrict__ subs, int ncs, int* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nact * ncs) return;
  const int j = t / ncs, q = t % ncs;
  const int b = list ? list[j] : j;
  const int m = b / nrhs, r = b % nrhs;
  out[t] = (m * nsub + subs[q]) * nrhs + r;
}

}  // namespace

template <typename T>
void launch_dd_gather(long long nl, int items_l, int nsub, int nrhs, long long ng, const int* map,
                      const typename CT<T>::type* res, typename CT<T>::type* out, cudaStream_t s) {
  k_dd_gather<<<dim3((unsigned)((nl + 255) / 256), sel_items(items_l)), 256, 0, s>>>(nl, nsub, nrhs, ng, map, res, out,
                                                                                   g_sel.list);
}
template <typename T>
void launch_dd_scatter(long long nl, int items_l, int nsub, int nrhs, long long ng, const int* map,
                       const typename CT<T>::type* xs, typename CT<T>::type* x, cudaStream_t s) {
  k_dd_scatter<<<dim3((unsigned)((nl + 255) / 256), sel_items(items_l)), 256, 0, s>>>(nl, nsub, nrhs, ng, map, xs, x,
                                                                                    g_sel.list);
}
void launch_expand_items(const int* list, int nact, int nrhs, int nsub, const int* subs, int ncs, int* out,
                         cudaStream_t s) {
  const int n = nact * ncs;
  k_expand_items<<<(n + 127) / 128, 128, 0, s>>>(list, nact, nrhs, nsub, subs, ncs, out);
}

template void launch_dd_gather<float>(long long, int, int, int, long long, const int*, const float2*, float2*, cudaStream_t);
template void launch_dd_gather<double>(long long, int, int, int, long long, const int*, const double2*, double2*, cudaStream_t);
template void launch_dd_scatter<float>(long long, int, int, int, long long, const int*, const float2*, float2*, cudaStream_t);
template void launch_dd_scatter<double>(long long, int, int, int, long long, const int*, const double2*, double2*, cudaStream_t);

}  // namespace ehs
