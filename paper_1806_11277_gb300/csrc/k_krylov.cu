// FP64 kernels of the flexible GMRES outer solve (Sec. 2.2: the shifted
// operator preconditions a flexible GMRES; Sec. 6: 1e-6 relative residual).
// Arnoldi uses classical Gram-Schmidt twice (CGS2); the dot products are
// reduced in a fixed order (per-block partials, then one warp per output with
// a fixed tree), so results are deterministic for a given launch shape.
#include "kernels.h"

namespace ehs {
namespace {

constexpr int KB = 256;      // threads per block
constexpr int MAXV = 12;     // max vectors per multi-dot (restart <= 11)

__device__ __forceinline__ double2 warp_sum(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-reduce nv complex accumulators and write part[(item*nv+i)*nblk+blk]
__device__ __forceinline__ void block_store(double2* acc, int nv, double2* part, int item, int nblk) {
  __shared__ double2 sh[KB / 32][MAXV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < nv; ++i) {
    double2 v = warp_sum(acc[i]);
    if (lane == 0) sh[wid][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double2 s = make_double2(0, 0);
    for (int w = 0; w < KB / 32; ++w) { s.x += sh[w][threadIdx.x].x; s.y += sh[w][threadIdx.x].y; }
    part[((long long)item * nv + threadIdx.x) * nblk + blockIdx.x] = s;
  }
}

__global__ void k_mdot(long long n, int items, int nv, const double2* __restrict__ V,
                       const double2* __restrict__ w, double2* part, int nblk) {
  const int item = blockIdx.y;
  double2 acc[MAXV];
  for (int i = 0; i < MAXV; ++i) acc[i] = make_double2(0, 0);
  const double2* wv = w + (long long)item * n;
  for (long long e = (long long)blockIdx.x * KB + threadIdx.x; e < n; e += (long long)nblk * KB) {
    const double2 we = __ldg(wv + e);
#pragma unroll
    for (int i = 0; i < MAXV; ++i) {
      if (i < nv) {
        const double2 v = __ldg(V + ((long long)i * items + item) * n + e);
        acc[i].x = fma(v.x, we.x, fma(v.y, we.y, acc[i].x));   // conj(v) * w
        acc[i].y = fma(v.x, we.y, fma(-v.y, we.x, acc[i].y));
      }
    }
  }
  block_store(acc, nv, part, item, nblk);
}

__global__ void k_mupdate(long long n, int items, int nv, const double2* __restrict__ V,
                          const double2* __restrict__ h, double2* __restrict__ w, double2* part,
                          int nblk, int dot, double* nrm_part) {
  const int item = blockIdx.y;
  double2 hh[MAXV];
  for (int i = 0; i < MAXV; ++i) hh[i] = i < nv ? h[(long long)item * nv + i] : make_double2(0, 0);
  double2 acc[MAXV];
  for (int i = 0; i < MAXV; ++i) acc[i] = make_double2(0, 0);
  double nacc = 0.0;
  double2* wv = w + (long long)item * n;
  for (long long e = (long long)blockIdx.x * KB + threadIdx.x; e < n; e += (long long)nblk * KB) {
    double2 we = wv[e];
    double2 vv[MAXV];
#pragma unroll
    for (int i = 0; i < MAXV; ++i) {
      if (i < nv) {
        vv[i] = __ldg(V + ((long long)i * items + item) * n + e);
        we.x -= vv[i].x * hh[i].x - vv[i].y * hh[i].y;
        we.y -= vv[i].x * hh[i].y + vv[i].y * hh[i].x;
      }
    }
    wv[e] = we;
    if (dot) {
#pragma unroll
      for (int i = 0; i < MAXV; ++i) {
        if (i < nv) {
          acc[i].x = fma(vv[i].x, we.x, fma(vv[i].y, we.y, acc[i].x));
          acc[i].y = fma(vv[i].x, we.y, fma(-vv[i].y, we.x, acc[i].y));
        }
      }
    }
    nacc = fma(we.x, we.x, fma(we.y, we.y, nacc));
  }
  if (dot) block_store(acc, nv, part, item, nblk);
  if (nrm_part) {
    __shared__ double shn[KB / 32];
    double v = warp_sum(nacc);
    if ((threadIdx.x & 31) == 0) shn[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < KB / 32; ++i) s += shn[i];
      nrm_part[(long long)item * nblk + blockIdx.x] = s;
    }
  }
}

__global__ void k_norm_part(long long n, const double2* __restrict__ w, double* part, int nblk) {
  const int item = blockIdx.y;
  const double2* wv = w + (long long)item * n;
  double nacc = 0.0;
  for (long long e = (long long)blockIdx.x * KB + threadIdx.x; e < n; e += (long long)nblk * KB) {
    const double2 we = __ldg(wv + e);
    nacc = fma(we.x, we.x, fma(we.y, we.y, nacc));
  }
  __shared__ double shn[KB / 32];
  double v = warp_sum(nacc);
  if ((threadIdx.x & 31) == 0) shn[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < KB / 32; ++i) s += shn[i];
    part[(long long)item * nblk + blockIdx.x] = s;
  }
}

// one warp per output: out[o] (+)= sum_blk part[o*nblk + blk]
__global__ void k_reduce_parts(int nout, int nblk, const double2* __restrict__ part, double2* out,
                               int accumulate) {
  const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= nout) return;
  double2 s = make_double2(0, 0);
  for (int b = lane; b < nblk; b += 32) {
    const double2 v = part[(long long)o * nblk + b];
    s.x += v.x; s.y += v.y;
  }
  s = warp_sum(s);
  if (lane == 0) {
    if (accumulate) { s.x += out[o].x; s.y += out[o].y; }
    out[o] = s;
  }
}
__global__ void k_reduce_norm(int items, int nblk, const double* __restrict__ part, double* out) {
  const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= items) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(long long)o * nblk + b];
  s = warp_sum(s);
  if (lane == 0) out[o] = sqrt(s);
}

__global__ void k_scale_inv(long long n, const double2* __restrict__ w, const double* __restrict__ nrm,
                            double2* __restrict__ out) {
  const int item = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double s = nrm[item] > 0.0 ? 1.0 / nrm[item] : 0.0;
  const double2 v = w[(long long)item * n + e];
  out[(long long)item * n + e] = make_double2(v.x * s, v.y * s);
}

__global__ void k_c128_c64(long long n, const double2* __restrict__ in, float2* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) { const double2 v = in[e]; out[e] = make_float2((float)v.x, (float)v.y); }
}
__global__ void k_c64_c128(long long n, const float2* __restrict__ in, double2* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) { const float2 v = in[e]; out[e] = make_double2(v.x, v.y); }
}

template <typename CZ>
__global__ void k_xupdate(long long n, int items, int m, const CZ* __restrict__ Z,
                          const double2* __restrict__ y, const int* __restrict__ kused,
                          double2* __restrict__ x) {
  const int item = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int k = kused[item];
  double2 acc = x[(long long)item * n + e];
  for (int i = 0; i < k; ++i) {
    const CZ z = Z[((long long)i * items + item) * n + e];
    const double2 yi = y[(long long)item * m + i];
    acc.x = fma((double)z.x, yi.x, fma(-(double)z.y, yi.y, acc.x));
    acc.y = fma((double)z.x, yi.y, fma((double)z.y, yi.x, acc.y));
  }
  x[(long long)item * n + e] = acc;
}

inline unsigned nb(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

int krylov_nblk(long long n) {
  long long b = (n + KB - 1) / KB;
  if (b > 2 * 152) b = 2 * 152;   // one wave per item at the reduction passes' 2 CTAs per SM (measured)
  return (int)(b < 1 ? 1 : b);
}

void launch_mdot(long long n, int items, int nv, const double2* V, const double2* w, double2* part,
                 int nblk, cudaStream_t s) {
  k_mdot<<<dim3(nblk, items), KB, 0, s>>>(n, items, nv, V, w, part, nblk);
}
void launch_mupdate(long long n, int items, int nv, const double2* V, const double2* h, double2* w,
                    double2* part, int nblk, int dot, double* nrm_part, cudaStream_t s) {
  k_mupdate<<<dim3(nblk, items), KB, 0, s>>>(n, items, nv, V, h, w, part, nblk, dot, nrm_part);
}
void launch_reduce_parts(int items, int nv, int nblk, const double2* part, double2* out,
                         int accumulate, cudaStream_t s) {
  const int nout = items * nv;
  k_reduce_parts<<<nb((long long)nout * 32, 128), 128, 0, s>>>(nout, nblk, part, out, accumulate);
}
void launch_norm_part(long long n, int items, const double2* w, double* part, int nblk, cudaStream_t s) {
  k_norm_part<<<dim3(nblk, items), KB, 0, s>>>(n, w, part, nblk);
}
void launch_reduce_norm(int items, int nblk, const double* part, double* out, cudaStream_t s) {
  k_reduce_norm<<<nb((long long)items * 32, 128), 128, 0, s>>>(items, nblk, part, out);
}
void launch_scale_inv(long long n, int items, const double2* w, const double* nrm, double2* out,
                      cudaStream_t s) {
  k_scale_inv<<<dim3(nb(n, 256), items), 256, 0, s>>>(n, w, nrm, out);
}
void launch_cast_c128_c64(long long n, const double2* in, float2* out, cudaStream_t s) {
  k_c128_c64<<<nb(n, 256), 256, 0, s>>>(n, in, out);
}
void launch_cast_c64_c128(long long n, const float2* in, double2* out, cudaStream_t s) {
  k_c64_c128<<<nb(n, 256), 256, 0, s>>>(n, in, out);
}
void launch_copy(long long nbytes, const void* in, void* out, cudaStream_t s) {
  cudaMemcpyAsync(out, in, nbytes, cudaMemcpyDeviceToDevice, s);
}
template <typename CZ>
void launch_xupdate(long long n, int items, int m, const CZ* Z, const double2* y, const int* kused,
                    double2* x, cudaStream_t s) {
  k_xupdate<CZ><<<dim3(nb(n, 256), items), 256, 0, s>>>(n, items, m, Z, y, kused, x);
}
template void launch_xupdate<float2>(long long, int, int, const float2*, const double2*, const int*,
                                     double2*, cudaStream_t);
template void launch_xupdate<double2>(long long, int, int, const double2*, const double2*, const int*,
                                      double2*, cudaStream_t);

}  // namespace ehs
