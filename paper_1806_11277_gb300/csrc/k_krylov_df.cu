// FP64-class (double-float) kernels of the outer FGMRES solve, its operator
// K (unshifted, Sec. 3 eq. elasticHelmReformulatedSystem), the true residual,
// and the coarsest-level solve.  Same algorithms as k_krylov.cu / k_fine.cu /
// k_dense.cu, carried out in df64 (see df64.cuh) on the FP32 pipe; the Arnoldi
// step is CGS2 (k_mdot_df, k_mupdate_df, k_update_scale_cast_df) or delayed
// CGS2 (k_mdot2_df, k_dupdate_df).
//
// Layouts: Krylov basis V and solution x as complex df64 (float4 per value),
// preconditioned directions Z as complex64 (the multigrid cycle's output
// precision), fine coefficients as 4 df64 reals per cell, coarsest inverse as
// complex df64.
#include "df64.cuh"
#include "kernels.h"

namespace ehs {

struct Coef4df {
  dfr mu, kap, mr, mi;
};

namespace {

constexpr int KB = 256;
constexpr int MAXV = 12;

__device__ __forceinline__ dfr shfl_df(dfr v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ dfc warp_sum_df(dfc v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.re = df_add(v.re, shfl_df(v.re, o));
    v.im = df_add(v.im, shfl_df(v.im, o));
  }
  return v;
}
__device__ __forceinline__ dfr warp_sum_df(dfr v) {
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, shfl_df(v, o));
  return v;
}

__device__ __forceinline__ dfc shfl_dfc(dfc v, int o) { return {shfl_df(v.re, o), shfl_df(v.im, o)}; }

// Block partials of NV sums.  The warp stage halves the values per lane at each
// exchange (reduce-scatter): at the exchange with lane ^ o a lane keeps one half
// of its values, sends the other and adds what it receives, so that after
// log2(P) exchanges (P = NV rounded up to a power of two) each value's sum over
// 32 / P lanes sits in one lane, and the remaining exchanges add across those.
// That moves P - 1 + log2(32 / P) values per lane instead of 5 NV.  The order of
// every sum is fixed by the lane indices, so the result does not depend on timing.
template <int NV>
__device__ __forceinline__ void block_store_df(const dfc* acc, float4* part, int item, int nblk) {
  constexpr int P = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : 16;
  static_assert(NV <= MAXV && MAXV <= 16, "sums per block");
  __shared__ dfc sh[KB / 32][MAXV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  dfc v[P];
#pragma unroll
  for (int k = 0; k < P; ++k) v[k] = k < NV ? acc[k] : dfc_zero();
  int idx = 0;
#pragma unroll
  for (int cnt = P, o = 16; cnt > 1; cnt >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < cnt / 2; ++k) {
      const dfc keep = up ? v[cnt / 2 + k] : v[k];
      const dfc send = up ? v[k] : v[cnt / 2 + k];
      v[k] = dfc_add(keep, shfl_dfc(send, o));
    }
    if (up) idx += cnt / 2;
  }
#pragma unroll
  for (int o = 16 / P; o > 0; o >>= 1) v[0] = dfc_add(v[0], shfl_dfc(v[0], o));
  if ((lane & (32 / P - 1)) == 0 && idx < NV) sh[wid][idx] = v[0];
  const int nv = NV;
  __syncthreads();
  if (threadIdx.x < nv) {
    dfc s = dfc_zero();
    for (int w = 0; w < KB / 32; ++w) s = dfc_add(s, sh[w][threadIdx.x]);
    dfc_st(part + ((long long)item * nv + threadIdx.x) * nblk + blockIdx.x, s);
  }
}
__device__ __forceinline__ void block_store_norm(dfr v, float2* part, int item, int nblk) {
  __shared__ dfr shn[KB / 32];
  v = warp_sum_df(v);
  if ((threadIdx.x & 31) == 0) shn[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    dfr s = df_zero();
    for (int i = 0; i < KB / 32; ++i) s = df_add(s, shn[i]);
    part[(long long)item * nblk + blockIdx.x] = make_float2(s.hi, s.lo);
  }
}

// Last-block reduction.  Every block of an item has written its partials; the
// block that finishes last for the item (counted in cnt[item], which it resets)
// sums them.  The sum runs in a fixed order -- per output, lanes stride over
// the blocks and a warp tree combines them, as k_reduce_parts_df does -- so the
// result is the same whichever block finishes last.  Partials are read with
// L1-bypassing loads (other blocks wrote them).
__device__ __forceinline__ bool last_block(int* cnt, int item, int nblk) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(cnt + item, 1) == nblk - 1;
  __syncthreads();
  return last;
}
__device__ __forceinline__ void reduce_dots_last(int item, int nv, int nblk, const float4* part, float4* out,
                                                 double2* outd, int* cnt) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < nv; i += KB / 32) {
    const long long o = (long long)item * nv + i;
    dfc s = dfc_zero();
    for (int b = lane; b < nblk; b += 32) {
      const float4 v = __ldcg(part + o * nblk + b);
      s = dfc_add(s, dfc{{v.x, v.z}, {v.y, v.w}});      // the storage order of dfc_st
    }
    s = warp_sum_df(s);
    if (lane == 0) {
      dfc_st(out + o, s);
      outd[o] = dfc_to_d2(s);
    }
  }
  if (threadIdx.x == 0) cnt[item] = 0;
}
__device__ __forceinline__ void reduce_norm_last(int item, int nblk, const float2* part, double* out, float2* inv,
                                                 int* cnt) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    dfr s = df_zero();
    for (int b = lane; b < nblk; b += 32) {
      const float2 v = __ldcg(part + (long long)item * nblk + b);
      s = df_add(s, {v.x, v.y});
    }
    s = warp_sum_df(s);
    if (lane == 0) {
      const double nrm = sqrt(df_to_d(s));   // one FP64 sqrt per item
      out[item] = nrm;
      const dfr iv = df_from_d(nrm > 0.0 ? 1.0 / nrm : 0.0);
      inv[item] = make_float2(iv.hi, iv.lo);
      cnt[item] = 0;
    }
  }
}

// Norm of w'' = w' - V h2 without forming it: with h2 = V^H w' and V orthonormal,
// ||w''||^2 = ||w'||^2 - ||h2||^2 (the neglected term is h2^H (V^H V - I) h2, of the
// order of the basis' loss of orthogonality times ||h2||^2, itself the square of a
// second-pass correction).  Sums the block partials of ||w'||^2 as reduce_norm_last
// does, subtracts the squares of the nv coefficients this block just wrote to h
// (df64), and stores the norm and its df64 inverse.
__device__ __forceinline__ void reduce_norm_pythag_last(int item, int nv, int nblk, const float2* part,
                                                        const float4* h, double* out, float2* inv) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    dfr s = df_zero();
    for (int b = lane; b < nblk; b += 32) {
      const float2 v = __ldcg(part + (long long)item * nblk + b);
      s = df_add(s, {v.x, v.y});
    }
    s = warp_sum_df(s);
    if (lane == 0) {
      for (int i = 0; i < nv; ++i) {
        const dfc hv = dfc_ldv(h + (long long)item * nv + i);   // written by this block
        s = df_sub(s, df_add(df_mul(hv.re, hv.re), df_mul(hv.im, hv.im)));
      }
      const double n2 = df_to_d(s);
      const double nrm = sqrt(n2 > 0.0 ? n2 : 0.0);   // one FP64 sqrt per item
      out[item] = nrm;
      const dfr iv = df_from_d(nrm > 0.0 ? 1.0 / nrm : 0.0);
      inv[item] = make_float2(iv.hi, iv.lo);
    }
  }
}

// The lane vectors dacc2_mfma takes for a coefficient h (df64 complex): (h.re, h.re) and
// (-h.im, h.im), high parts then low parts, as two float4.
__device__ __forceinline__ void load_hpairs(const float4* hp, float4* out) {
  const dfc hv = dfc_ldv(hp);
  out[0] = make_float4(hv.re.hi, hv.re.hi, hv.re.lo, hv.re.lo);
  out[1] = make_float4(-hv.im.hi, hv.im.hi, -hv.im.lo, hv.im.lo);
}

// partial dots conj(V_i) . w per block; with cnt, the last block of each item also forms
// the sums (out: df64, outd: double copy for the host)
template <int NV>
__global__ void __launch_bounds__(KB, 2) k_mdot_df(long long n, int items, const float4* __restrict__ V,
                                                const float4* __restrict__ w, float4* part, int nblk,
                                                const int* __restrict__ il, int* cnt, float4* out, double2* outd) {
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  dacc2 acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = dacc2_zero();
  const float4* wv = w + (long long)item * n;
  for (long long e = (long long)blockIdx.x * KB + threadIdx.x; e < n; e += (long long)nblk * KB) {
    // every load of the element first: NV + 1 independent 16-byte loads in flight per thread
    dfc vv[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) vv[i] = dfc_ld(V + ((long long)i * items + item) * n + e);
    const dfc we = dfc_ld(wv + e);
    const float2 wah = make_float2(we.re.hi, -we.re.hi), wal = make_float2(we.re.lo, -we.re.lo);
    const float2 wbh = make_float2(we.im.hi, we.im.hi), wbl = make_float2(we.im.lo, we.im.lo);
#pragma unroll
    for (int i = 0; i < NV; ++i) dacc2_cfma(acc[i], dfc2_of(vv[i]), wah, wal, wbh, wbl);
  }
  dfc vals[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) vals[i] = dacc2_val(acc[i]);
  block_store_df<NV>(vals, part, item, nblk);
  if (cnt && last_block(cnt, item, nblk)) reduce_dots_last(item, NV, nblk, part, out, outd, cnt);
}

// w -= sum_i V_i h_i (stored unless store = 0); optional partial dots of V with the new w and |w|^2.
// With cnt, the last block of each item also forms the dots' sums (out, outd)
// and/or the norm (nrm, inv = 1/norm): with both, the norm of the vector that
// removing V out from w would leave (reduce_norm_pythag_last).
// h sits in shared memory and the dot pass re-reads V_i (an L1 hit: the block
// read it a moment earlier), which keeps the kernel at two blocks per SM.
template <int NV>
__global__ void __launch_bounds__(KB, 2) k_mupdate_df(long long n, int items, const float4* __restrict__ V,
                                                      const float4* __restrict__ h, float4* __restrict__ w,
                                                      float4* part, int nblk, int dot, float2* nrm_part,
                                                      const int* __restrict__ il, int* cnt, float4* out,
                                                      double2* outd, double* nrm, float2* inv, int store) {
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  __shared__ float4 hs[NV][2];
  if (threadIdx.x < NV) load_hpairs(h + (long long)item * NV + threadIdx.x, hs[threadIdx.x]);
  __syncthreads();
  dacc2 acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = dacc2_zero();
  dacc nacc = dacc_zero();
  float4* wv = w + (long long)item * n;
  for (long long e = (long long)blockIdx.x * KB + threadIdx.x; e < n; e += (long long)nblk * KB) {
    dacc2 sv = dacc2_zero();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float4 a = hs[i][0], b = hs[i][1];
      dacc2_mfma(sv, dfc2_of(dfc_ld(V + ((long long)i * items + item) * n + e)), make_float2(a.x, a.y),
                 make_float2(a.z, a.w), make_float2(b.x, b.y), make_float2(b.z, b.w));
    }
    const dfc we = dfc_sub(dfc_ldv(wv + e), dacc2_val(sv));
    if (store) dfc_st(wv + e, we);
    if (dot) {
      const float2 wah = make_float2(we.re.hi, -we.re.hi), wal = make_float2(we.re.lo, -we.re.lo);
      const float2 wbh = make_float2(we.im.hi, we.im.hi), wbl = make_float2(we.im.lo, we.im.lo);
#pragma unroll
      for (int i = 0; i < NV; ++i)
        dacc2_cfma(acc[i], dfc2_of(dfc_ld(V + ((long long)i * items + item) * n + e)), wah, wal, wbh, wbl);
    }
    dacc_fma(nacc, we.re, we.re);
    dacc_fma(nacc, we.im, we.im);
  }
  if (dot) {
    dfc vals[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) vals[i] = dacc2_val(acc[i]);
    block_store_df<NV>(vals, part, item, nblk);
  }
  if (nrm_part) block_store_norm(dacc_val(nacc), nrm_part, item, nblk);
  if (cnt && (dot || nrm_part) && last_block(cnt, item, nblk)) {
    if (dot) reduce_dots_last(item, NV, nblk, part, out, outd, cnt);
    if (dot && nrm_part) {
      __syncthreads();                              // the dots' sums are in out
      reduce_norm_pythag_last(item, NV, nblk, nrm_part, out, nrm, inv);
    } else if (nrm_part) {
      reduce_norm_last(item, nblk, nrm_part, nrm, inv, cnt);
    }
  }
}

// The last pass of an Arnoldi step: V_{j+1} = (w - sum_i V_i (h0_i + h_i)) * inv (df64)
// and its complex64 copy, the next preconditioner input; w itself is not written.
template <int NV>
__global__ void __launch_bounds__(KB, 3) k_update_scale_cast_df(long long n, int items, const float4* __restrict__ V,
                                                                const float4* __restrict__ h0,
                                                                const float4* __restrict__ h,
                                                                const float4* __restrict__ w,
                                                                const float2* __restrict__ inv,
                                                                float4* __restrict__ out, float2* __restrict__ out32,
                                                                int nblk, const int* __restrict__ il) {
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  __shared__ float4 hs[NV];
  if (threadIdx.x < NV) {   // the coefficients h0 + h (h0 may be null)
    dfc hv = dfc_ldv(h + (long long)item * NV + threadIdx.x);
    if (h0) hv = dfc_add(dfc_ldv(h0 + (long long)item * NV + threadIdx.x), hv);
    dfc_st(hs + threadIdx.x, hv);
  }
  __syncthreads();
  const float2 sc = inv[item];
  const dfr iv = {sc.x, sc.y};
  const float4* wv = w + (long long)item * n;
  // scalar Dot2 steps here: this pass is bound by memory, and the paired form's extra
  // shared-memory operands measured slower at large nv
  for (long long e = (long long)blockIdx.x * KB + threadIdx.x; e < n; e += (long long)nblk * KB) {
    dcacc sv = dcacc_zero();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float4 hv = hs[i];   // the storage order of dfc_st
      dcacc_fma(sv, dfc_ld(V + ((long long)i * items + item) * n + e), dfc{{hv.x, hv.z}, {hv.y, hv.w}});
    }
    const dfc v = dfc_scale(dfc_sub(dfc_ld(wv + e), dcacc_val(sv)), iv);
    dfc_st(out + (long long)item * n + e, v);
    out32[(long long)item * n + e] = dfc_to_f2(v);
  }
}

// ---- delayed CGS2 (one dot pass and one update pass per Arnoldi step) --------
// Step j starts with v_0..v_{j-1} orthonormal and, in slot j, u_j: the direction the
// preconditioner was applied to, orthogonalised once and scaled by the norm that
// assumed the first pass exact.  With z_j = M^{-1} u_j and w = K z_j, one pass over
// the basis gives a = V^H u_j, b = V^H w, u_j^H w, ||u_j||^2 and ||w||^2; from them
//   v_j     = (u_j - V a) / sigma,          sigma = sqrt(||u_j||^2 - ||a||^2),
//   h_j     = v_j^H w = (u_j^H w - a^H b) / sigma,
//   u_{j+1} = (w - V b - v_j h_j) / rho,    rho = sqrt(||w||^2 - ||b||^2 - |h_j|^2),
// the second pass of Gram-Schmidt for u_j riding on the first pass for w.  Column j
// of the Hessenberg matrix is (b, h_j, rho); the next step replaces its
// subdiagonal by rho * sigma_{j+1} and adds rho * a_{j+1} above it (K z_j = w and
// rho u_{j+1} = V_{j+1} a_{j+1} + rho sigma_{j+1} v_{j+1}).  In exact arithmetic
// the basis and the Hessenberg matrix are those of CGS2; the preconditioner sees
// u_j instead of v_j, which flexible GMRES allows (its space is spanned by the z_j
// actually formed).

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zcmul(double2 a, double2 b) {   // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// First pass of step j = NS - 1 (slots 0..j of V, slot j holding u_j).  Blocks
// 2k and 2k + 1 of an item cover the same elements: the even block forms
// conj(V_i) u_j for i <= j (i = j: ||u_j||^2) as compensated Dot2 sums, the odd
// one conj(V_i) w (i = j: u_j^H w) and ||w||^2 from FP32 products of the high
// parts; running side by side, the second read of the basis is an L2 hit.  Only
// the second projection (a, sigma) has to be exact to double-float: b, u_j^H w
// and ||w||^2 fix what the update subtracts from w, the Hessenberg column records
// exactly that, and the next step's a measures (and its update removes) whatever
// their rounding left along the basis, as the second pass of CGS2 does for the
// first; rho only scales u_{j+1} (sigma of the next step measures its norm) and
// the step's residual estimate.  The last block of the item sums the partials
// (fixed order, as reduce_dots_last) and forms the update coefficients in FP64:
//   coef[item * KDS + ...]  (df64)  a_0..a_{j-1}, b_i - a_i h_j / sigma (i < j),
//                                   h_j / sigma, 1 / sigma, 1 / rho
//   outd[item * KDS + ...]  (FP64)  a_0..a_{j-1}, sigma, b_0..b_{j-1}, h_j, rho
// (sigma = 1 and no a at j = 0: u_0 = r / ||r|| is normalised by the norm pass).
template <int NS>
__global__ void __launch_bounds__(KB, 2) k_mdot2_df(long long n, int items, const float4* __restrict__ V,
                                                 const float4* __restrict__ w, float4* part, int nblk,
                                                 const int* __restrict__ il, int* cnt, float4* coef, double2* outd) {
  constexpr int NO = NS + 1;   // NS dots and one norm per half
  static_assert(NO <= MAXV, "sums per half");
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const int half = blockIdx.x & 1, blk = blockIdx.x >> 1;
  dfc vals[NO];
  if (half) {
    // first projection of w: FP32 products of the high parts, FP32 sums over the thread's ~10
    // elements, df64 from the block sums on
    const float2* wv = (const float2*)(w + (long long)item * n);   // (re.hi, im.hi) of each value
    float2 af[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) af[i] = make_float2(0.f, 0.f);
    float nf = 0.f;
    for (long long e = (long long)blk * KB + threadIdx.x; e < n; e += (long long)nblk * KB) {
      const float2 x = __ldg(wv + 2 * e);
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        const float2 v = __ldg((const float2*)(V + ((long long)i * items + item) * n + e));
        af[i].x = fmaf(v.x, x.x, fmaf(v.y, x.y, af[i].x));    // conj(v) * x
        af[i].y = fmaf(v.x, x.y, fmaf(-v.y, x.x, af[i].y));
      }
      nf = fmaf(x.x, x.x, fmaf(x.y, x.y, nf));
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) vals[i] = {df_from_f(af[i].x), df_from_f(af[i].y)};
    vals[NS] = {df_from_f(nf), df_zero()};
  } else {
    // second projection of u_j (and ||u_j||^2): compensated Dot2 sums of the df64 values
    dacc2 acc[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) acc[i] = dacc2_zero();
    for (long long e = (long long)blk * KB + threadIdx.x; e < n; e += (long long)nblk * KB) {
      dfc vv[NS];
#pragma unroll
      for (int i = 0; i < NS; ++i) vv[i] = dfc_ld(V + ((long long)i * items + item) * n + e);
      const dfc xe = vv[NS - 1];
      const float2 wah = make_float2(xe.re.hi, -xe.re.hi), wal = make_float2(xe.re.lo, -xe.re.lo);
      const float2 wbh = make_float2(xe.im.hi, xe.im.hi), wbl = make_float2(xe.im.lo, xe.im.lo);
#pragma unroll
      for (int i = 0; i < NS; ++i) dacc2_cfma(acc[i], dfc2_of(vv[i]), wah, wal, wbh, wbl);
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) vals[i] = dacc2_val(acc[i]);
    vals[NS] = dfc_zero();
  }
  block_store_df<NO>(vals, part, item, 2 * nblk);
  if (!cnt || !last_block(cnt, item, 2 * nblk)) return;
  __shared__ double2 sd[2 * NO];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = wid; o < 2 * NO; o += KB / 32) {
    const int hf = o / NO, oo = o - hf * NO;
    const float4* p = part + ((long long)item * NO + oo) * (2 * nblk) + hf;
    dfc s = dfc_zero();
    for (int b = lane; b < nblk; b += 32) {
      const float4 v = __ldcg(p + 2 * b);
      s = dfc_add(s, dfc{{v.x, v.z}, {v.y, v.w}});   // the storage order of dfc_st
    }
    s = warp_sum_df(s);
    if (lane == 0) sd[o] = dfc_to_d2(s);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  constexpr int j = NS - 1;
  const double2* A = sd;        // A[i] = V_i^H u_j (i < j), A[j].x = ||u_j||^2
  const double2* B = sd + NO;   // B[i] = V_i^H w (i < j), B[j] = u_j^H w, B[NS].x = ||w||^2
  double sig = 1.0;
  if (j > 0) {
    double s2 = A[j].x;
    for (int i = 0; i < j; ++i) s2 -= A[i].x * A[i].x + A[i].y * A[i].y;
    sig = s2 > 0.0 ? sqrt(s2) : 0.0;
  }
  const double isig = sig > 0.0 ? 1.0 / sig : 0.0;
  double2 hj = B[j];
  for (int i = 0; i < j; ++i) {
    const double2 t = zcmul(A[i], B[i]);
    hj.x -= t.x;
    hj.y -= t.y;
  }
  hj.x *= isig;
  hj.y *= isig;
  double r2 = B[NS].x - (hj.x * hj.x + hj.y * hj.y);
  for (int i = 0; i < j; ++i) r2 -= B[i].x * B[i].x + B[i].y * B[i].y;
  // r2 carries the first projection's FP32 rounding (about 1e-7 of ||w||^2): below 1e-12 ||w||^2 it
  // says nothing, and any positive scale serves (sigma of the next step measures the true norm)
  const double r2min = 1e-12 * B[NS].x;
  const double rho = sqrt(r2 > r2min ? r2 : r2min);
  const double2 cu = make_double2(hj.x * isig, hj.y * isig);
  float4* cf = coef + (long long)item * KDS;
  double2* od = outd + (long long)item * KDS;
  for (int i = 0; i < j; ++i) {
    const double2 t = zmul(A[i], cu);
    dfc_st(cf + i, dfc_from_d2(A[i]));
    dfc_st(cf + j + i, dfc_from_d2(make_double2(B[i].x - t.x, B[i].y - t.y)));
    od[i] = A[i];
    od[j + 1 + i] = B[i];
  }
  dfc_st(cf + 2 * j, dfc_from_d2(cu));
  dfc_st(cf + 2 * j + 1, dfc_from_d2(make_double2(isig, 0.0)));
  dfc_st(cf + 2 * j + 2, dfc_from_d2(make_double2(rho > 0.0 ? 1.0 / rho : 0.0, 0.0)));
  od[j] = make_double2(sig, 0.0);
  od[2 * j + 1] = hj;
  od[2 * j + 2] = make_double2(rho, 0.0);
  cnt[item] = 0;
}

// Second pass of step j = NJ: v_j = (u_j - sum_i V_i a_i) / sigma over slot j and
// u_{j+1} = (w - sum_i V_i c_i - u_j h_j / sigma) / rho into slot j + 1 with its
// complex64 copy (the next preconditioner input), c_i = b_i - a_i h_j / sigma;
// coefficients as k_mdot2_df stores them.  Slots below j are only read.
template <int NJ>
__global__ void __launch_bounds__(KB, 3) k_dupdate_df(long long n, int items, const float4* V, float4* vj,
                                                   float4* vn, const float4* __restrict__ w,
                                                   const float4* __restrict__ coef, float2* __restrict__ out32,
                                                   const int* __restrict__ il) {
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  constexpr int NC = 2 * NJ + 3;
  static_assert(NC <= KDS, "coefficients per item");
  __shared__ float4 cs[NC];
  if (threadIdx.x < NC) cs[threadIdx.x] = coef[(long long)item * KDS + threadIdx.x];
  __syncthreads();
  const float4 s4 = cs[2 * NJ + 1], r4 = cs[2 * NJ + 2];
  const dfr isig = {s4.x, s4.z}, irho = {r4.x, r4.z};
  const float4 u4 = cs[2 * NJ];
  const dfc cu = {{u4.x, u4.z}, {u4.y, u4.w}};
  const long long off = (long long)item * n;
  const float4* wv = w + off;
  float4* uv = vj + off;
  float4* nv = vn + off;
  for (long long e = (long long)blockIdx.x * KB + threadIdx.x; e < n; e += (long long)gridDim.x * KB) {
    dcacc sv = dcacc_zero(), sw = dcacc_zero();
#pragma unroll
    for (int i = 0; i < NJ; ++i) {
      const dfc vi = dfc_ld(V + ((long long)i * items + item) * n + e);
      const float4 a = cs[i], c = cs[NJ + i];   // the storage order of dfc_st
      dcacc_fma(sv, vi, dfc{{a.x, a.z}, {a.y, a.w}});
      dcacc_fma(sw, vi, dfc{{c.x, c.z}, {c.y, c.w}});
    }
    const dfc u = dfc_ldv(uv + e);      // rewritten below by this thread only
    dcacc_fma(sw, u, cu);
    if (NJ > 0) dfc_st(uv + e, dfc_scale(dfc_sub(u, dcacc_val(sv)), isig));
    const dfc x = dfc_scale(dfc_sub(dfc_ld(wv + e), dcacc_val(sw)), irho);
    dfc_st(nv + e, x);
    out32[off + e] = dfc_to_f2(x);
  }
}

__global__ void k_norm_part_df(long long n, const float4* __restrict__ w, float2* part, int nblk, const int* __restrict__ il) {
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const float4* wv = w + (long long)item * n;
  dacc nacc = dacc_zero();
  for (long long e = (long long)blockIdx.x * KB + threadIdx.x; e < n; e += (long long)nblk * KB) {
    const dfc we = dfc_ld(wv + e);
    dacc_fma(nacc, we.re, we.re);
    dacc_fma(nacc, we.im, we.im);
  }
  block_store_norm(dacc_val(nacc), part, item, nblk);
}

// one warp per output; writes the df64 value and its double copy for the host
__global__ void k_reduce_parts_df(int nout, int nblk, const float4* __restrict__ part, float4* out,
                                  double2* outd, int nv, const int* __restrict__ il) {
  const int oo = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (oo >= nout) return;
  const int o = il ? il[oo / nv] * nv + oo % nv : oo;
  dfc s = dfc_zero();
  for (int b = lane; b < nblk; b += 32) s = dfc_add(s, dfc_ld(part + (long long)o * nblk + b));
  s = warp_sum_df(s);
  if (lane == 0) {
    dfc_st(out + o, s);
    outd[o] = dfc_to_d2(s);
  }
}
// norm = sqrt(sum); writes the double norm for the host and 1/norm in df64
__global__ void k_reduce_norm_df(int items, int nblk, const float2* __restrict__ part, double* out,
                                 float2* inv, const int* __restrict__ il) {
  const int oo = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (oo >= items) return;
  const int o = il ? il[oo] : oo;
  dfr s = df_zero();
  for (int b = lane; b < nblk; b += 32) {
    const float2 v = part[(long long)o * nblk + b];
    s = df_add(s, {v.x, v.y});
  }
  s = warp_sum_df(s);
  if (lane == 0) {
    const double nrm = sqrt(df_to_d(s));   // one FP64 sqrt per item
    out[o] = nrm;
    const dfr iv = df_from_d(nrm > 0.0 ? 1.0 / nrm : 0.0);
    if (inv) inv[o] = make_float2(iv.hi, iv.lo);
  }
}

__global__ void k_scale_df(long long n, const float4* __restrict__ w, const float2* __restrict__ inv,
                           float4* __restrict__ out, const int* __restrict__ il) {
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float2 s = inv[item];
  dfc_st(out + (long long)item * n + e, dfc_scale(dfc_ld(w + (long long)item * n + e), {s.x, s.y}));
}

// V_j = w / ||w|| (df64) and its complex64 copy, the input of the preconditioner
__global__ void k_scale_cast_df(long long n, const float4* __restrict__ w, const float2* __restrict__ inv,
                                float4* __restrict__ out, float2* __restrict__ out32, const int* __restrict__ il) {
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float2 s = inv[item];
  const dfc v = dfc_scale(dfc_ld(w + (long long)item * n + e), {s.x, s.y});
  dfc_st(out + (long long)item * n + e, v);
  out32[(long long)item * n + e] = dfc_to_f2(v);
}

__global__ void k_xupdate_df(long long n, int items, int m, const float2* __restrict__ Z,
                             const float4* __restrict__ y, const int* __restrict__ kused,
                             float4* __restrict__ x) {
  const int item = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int k = kused[item];
  dfc acc = dfc_ldv(x + (long long)item * n + e);
  for (int i = 0; i < k; ++i)
    acc = dfc_add(acc, dfc_mulf(dfc_ld(y + (long long)item * m + i),
                                __ldg(Z + ((long long)i * items + item) * n + e)));
  dfc_st(x + (long long)item * n + e, acc);
}

__global__ void k_d2_to_df(long long n, const double2* __restrict__ in, float4* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dfc_st(out + e, dfc_from_d2(in[e]));
}
__global__ void k_df_to_d2(long long n, const float4* __restrict__ in, double2* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = dfc_to_d2(dfc_ld(in + e));
}
__global__ void k_df_to_f2(long long n, const float4* __restrict__ in, float2* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = dfc_to_f2(dfc_ld(in + e));
}
__global__ void k_coef_df(long long n, const Coef4<double>* __restrict__ in, Coef4df* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const Coef4<double> v = in[e];
  out[e] = {df_from_d(v.mu), df_from_d(v.kap), df_from_d(v.mr), df_from_d(v.mi)};
}

// --- FP64-class fine operator --------------------------------------------
template <typename V> __device__ __forceinline__ dfc ldx(const V* p, long long i);
template <> __device__ __forceinline__ dfc ldx<float4>(const float4* p, long long i) { return dfc_ld(p + i); }
template <> __device__ __forceinline__ dfc ldx<float2>(const float2* p, long long i) {
  return dfc_from_f2(__ldg(p + i));
}
__device__ __forceinline__ Coef4df ldcf_df(const Coef4df* p, long long c) {
  const float4* q = reinterpret_cast<const float4*>(p) + 2 * c;
  const float4 a = __ldg(q), b = __ldg(q + 1);
  return {{a.x, a.y}, {a.z, a.w}, {b.x, b.y}, {b.z, b.w}};
}

struct FinePdf {
  dfr h2inv, hinv, alpha;
};

template <typename V, int D>
__device__ __forceinline__ dfc row_u_df(const Grid& g, int k, long long c, const int i[3],
                                        const Coef4df* cf, const V* xk, const V* p, const FinePdf& P) {
  const long long sk = stride_of(g, k);
  const Coef4df c0 = ldcf_df(cf, c), c1 = ldcf_df(cf, c - sk);
  const dfc xc = ldx<V>(xk, c);
  dfc nb = dfc_zero();
  if (i[k] + 1 < g.n[k]) nb = dfc_add(nb, dfc_scale(ldx<V>(xk, c + sk), c0.mu));
  if (i[k] - 1 >= 1) nb = dfc_add(nb, dfc_scale(ldx<V>(xk, c - sk), c1.mu));
  const dfr base = df_add(c0.mu, c1.mu);
  dfr wsum = base;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j == k) continue;
    const long long sj = stride_of(g, j);
    const bool hp = i[j] + 1 < g.n[j], hm = i[j] - 1 >= 0;
    const long long cp = hp ? c + sj : c, cm = hm ? c - sj : c;
    dfr wp = df_add(base, df_add(ldcf_df(cf, cp).mu, ldcf_df(cf, cp - sk).mu));
    dfr wm = df_add(base, df_add(ldcf_df(cf, cm).mu, ldcf_df(cf, cm - sk).mu));
    wp = {wp.hi * 0.25f, wp.lo * 0.25f};   // exact scaling by a power of two
    wm = {wm.hi * 0.25f, wm.lo * 0.25f};
    wsum = df_add(wsum, df_add(wp, wm));
    if (hp) nb = dfc_add(nb, dfc_scale(ldx<V>(xk, c + sj), wp));
    if (hm) nb = dfc_add(nb, dfc_scale(ldx<V>(xk, c - sj), wm));
  }
  dfr rf = df_add(c0.mr, c1.mr), gf = df_add(c0.mi, c1.mi);
  rf = {rf.hi * 0.5f, rf.lo * 0.5f};
  gf = {gf.hi * 0.5f, gf.lo * 0.5f};
  const dfc dg = {df_sub(df_mul(wsum, P.h2inv), rf), df_add(gf, df_mul(P.alpha, rf))};
  dfc y = dfc_sub(dfc_mul(dg, xc), dfc_scale(nb, P.h2inv));
  return dfc_add(y, dfc_scale(dfc_sub(ldx<V>(p, c), ldx<V>(p, c - sk)), P.hinv));
}

template <typename V, int D>
__device__ __forceinline__ dfc row_p_df(const Grid& g, long long c, const int i[3], const Coef4df& c0,
                                        const V* x, const FinePdf& P) {
  const long long N = g.ncell;
  const dfc pc = ldx<V>(x + (long long)D * N, c);
  dfc s = dfc_zero();
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const V* xk = x + (long long)k * N;
    if (i[k] >= 1) s = dfc_add(s, ldx<V>(xk, c));
    if (i[k] + 1 < g.n[k]) s = dfc_sub(s, ldx<V>(xk, c + stride_of(g, k)));
  }
  return dfc_sub(dfc_scale(s, P.hinv), dfc_scale(pc, c0.kap));
}

// Setup-time tables of the 2D operator K (unshifted): per cell the diagonals of its
// low u_0 and u_1 face rows (complex df64, [set][2][ncell]; entries on Dirichlet
// faces are formed but never used) and per vertex ((nx + 1) (ny + 1)) the mean of mu
// over the four cells around it (df64, [set][vertex]; clamped at the edges, as the
// rows' tangential weights clamp), formed in FP64 from the FP64 coefficients.
__device__ __forceinline__ const Coef4<double>& cf_cl(const Coef4<double>* cf, int x, int y, int nx, int ny) {
  return cf[min(max(y, 0), ny - 1) * nx + min(max(x, 0), nx - 1)];
}
__device__ __forceinline__ double vm_d(const Coef4<double>* cf, int vx, int vy, int nx, int ny) {
  return 0.25 * ((cf_cl(cf, vx, vy, nx, ny).mu + cf_cl(cf, vx - 1, vy, nx, ny).mu) + cf_cl(cf, vx, vy - 1, nx, ny).mu +
                 cf_cl(cf, vx - 1, vy - 1, nx, ny).mu);
}
__global__ void k_apply_df_tables(Grid g, const Coef4<double>* __restrict__ cf, double h2inv, float4* __restrict__ dg,
                                  float2* __restrict__ vm) {
  const int nx = g.n[0], ny = g.n[1];
  const int nv = (nx + 1) * (ny + 1);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv) return;
  const int set = blockIdx.y;
  const Coef4<double>* cs = cf + (long long)set * g.ncell;
  const int vx = t % (nx + 1), vy = t / (nx + 1);
  const dfr v = df_from_d(vm_d(cs, vx, vy, nx, ny));
  vm[(long long)set * nv + t] = make_float2(v.hi, v.lo);
  if (vx >= nx || vy >= ny) return;
  const Coef4<double>& c0 = cf_cl(cs, vx, vy, nx, ny);
  // u_0 face between cells (vx-1, vy) and (vx, vy); u_1 face between (vx, vy-1) and (vx, vy)
  for (int k = 0; k < 2; ++k) {
    const Coef4<double>& c1 = k == 0 ? cf_cl(cs, vx - 1, vy, nx, ny) : cf_cl(cs, vx, vy - 1, nx, ny);
    const double wp = k == 0 ? vm_d(cs, vx, vy + 1, nx, ny) : vm_d(cs, vx + 1, vy, nx, ny);
    const double wsum = (c0.mu + c1.mu) + wp + vm_d(cs, vx, vy, nx, ny);
    const double rf = 0.5 * (c0.mr + c1.mr), gf = 0.5 * (c0.mi + c1.mi);
    dfc_st(dg + ((long long)set * 2 + k) * g.ncell + (long long)vy * nx + vx,
           dfc_from_d2(make_double2(wsum * h2inv - rf, gf)));
  }
}

// The 2D rows of K (alpha = 0) with the tables above: a u_k row at cell c is
// dg_k(c) x_c - (mu_c x_{c+e_k} + mu_{c-e_k} x_{c-e_k} + vm+ x_{c+e_j} + vm- x_{c-e_j}) / h^2
// + (p_c - p_{c-e_k}) / h, the same terms k_fine_apply_df forms from the cells'
// coefficients.  y = K x (mode 0) or b - K x (mode 1).
template <typename V>
__global__ void k_fine_apply_df2t(Grid g, int nrhs, const Coef4df* __restrict__ cf, const float4* __restrict__ dg,
                                  const float2* __restrict__ vmt, FinePdf P, const V* __restrict__ x,
                                  const float4* __restrict__ b, float4* __restrict__ y, int mode,
                                  const int* __restrict__ il) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const long long N = g.ncell;
  const int nx = g.n[0], ny = g.n[1];
  const long long vo = (long long)item * 3 * N;
  const int set = item / nrhs;
  const Coef4df* cs = cf + (long long)set * N;
  const float2* vms = vmt + (long long)set * (nx + 1) * (ny + 1);
  const V* xv = x + vo;
  const V* pv = xv + 2 * N;
  const int ix = (int)(c % nx), iy = (int)(c / nx);
  const Coef4df c0 = ldcf_df(cs, c);
  const float2 v00 = __ldg(vms + (long long)iy * (nx + 1) + ix);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    dfc r = dfc_zero();
    const int ik = k == 0 ? ix : iy, nk = k == 0 ? nx : ny;
    if (ik >= 1) {
      const long long sk = k == 0 ? 1 : nx, sj = k == 0 ? nx : 1;
      const int ij = k == 0 ? iy : ix, nj = k == 0 ? ny : nx;
      const V* xk = xv + (long long)k * N;
      const dfr mu1 = ldcf_df(cs, c - sk).mu;
      const float2 vp = __ldg(vms + (k == 0 ? (long long)(iy + 1) * (nx + 1) + ix : (long long)iy * (nx + 1) + ix + 1));
      dfc nb = dfc_zero();
      if (ik + 1 < nk) nb = dfc_add(nb, dfc_scale(ldx<V>(xk, c + sk), c0.mu));
      if (ik - 1 >= 1) nb = dfc_add(nb, dfc_scale(ldx<V>(xk, c - sk), mu1));
      if (ij + 1 < nj) nb = dfc_add(nb, dfc_scale(ldx<V>(xk, c + sj), dfr{vp.x, vp.y}));
      if (ij - 1 >= 0) nb = dfc_add(nb, dfc_scale(ldx<V>(xk, c - sj), dfr{v00.x, v00.y}));
      const dfc d = dfc_ld(dg + ((long long)set * 2 + k) * N + c);
      r = dfc_sub(dfc_mul(d, ldx<V>(xk, c)), dfc_scale(nb, P.h2inv));
      r = dfc_add(r, dfc_scale(dfc_sub(ldx<V>(pv, c), ldx<V>(pv, c - sk)), P.hinv));
      if (mode) r = dfc_sub(dfc_ld(b + vo + (long long)k * N + c), r);
    }
    dfc_st(y + vo + (long long)k * N + c, r);
  }
  const int i[3] = {ix, iy, 0};
  dfc r = row_p_df<V, 2>(g, c, i, c0, xv, P);
  if (mode) r = dfc_sub(dfc_ld(b + vo + 2 * N + c), r);
  dfc_st(y + vo + 2 * N + c, r);
}

// y = K x (mode 0) or y = b - K x (mode 1); x of type V, b and y complex df64
template <typename V, int D>
__global__ void k_fine_apply_df(Grid g, int nrhs, const Coef4df* __restrict__ cf, FinePdf P,
                                const V* __restrict__ x, const float4* __restrict__ b,
                                float4* __restrict__ y, int mode, const int* __restrict__ il) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const long long N = g.ncell;
  const long long vo = (long long)item * (D + 1) * N;
  const Coef4df* cs = cf + (long long)(item / nrhs) * N;
  const V* xv = x + vo;
  int i[3];
  cell_coords(g, c, i);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    dfc r = dfc_zero();
    if (i[k] >= 1) {
      r = row_u_df<V, D>(g, k, c, i, cs, xv + (long long)k * N, xv + (long long)D * N, P);
      if (mode) r = dfc_sub(dfc_ld(b + vo + (long long)k * N + c), r);
    }
    dfc_st(y + vo + (long long)k * N + c, r);
  }
  dfc r = row_p_df<V, D>(g, c, i, ldcf_df(cs, c), xv, P);
  if (mode) r = dfc_sub(dfc_ld(b + vo + (long long)D * N + c), r);
  dfc_st(y + vo + (long long)D * N + c, r);
}

// coarsest: x = Ainv r with Ainv in complex df64, r and x complex64; one warp per row
__global__ void k_dense_apply_df(int N, int nrhs, const float4* __restrict__ inv,
                                 const float2* __restrict__ r, float2* __restrict__ x,
                                 const int* __restrict__ il) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  if (warp >= N) return;
  const float4* row = inv + ((long long)(item / nrhs) * N + warp) * N;
  const float2* rv = r + (long long)item * N;
  dfc acc = dfc_zero();
  for (int j = lane; j < N; j += 32) acc = dfc_add(acc, dfc_mulf(dfc_ld(row + j), __ldg(rv + j)));
  acc = warp_sum_df(acc);
  if (lane == 0) x[(long long)item * N + warp] = dfc_to_f2(acc);
}

inline unsigned nb(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

FinePdf mkPdf(double h, double alpha) {
  FinePdf P;
  auto split = [](double v) {
    dfr r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
  };
  P.h2inv = split(1.0 / (h * h));
  P.hinv = split(1.0 / h);
  P.alpha = split(alpha);
  return P;
}

}  // namespace

#define EHS_NV_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11)
void launch_mdot_df(long long n, int items, int nv, const float4* V, const float4* w, float4* part,
                    int nblk, cudaStream_t s, int* cnt, float4* out, double2* outd) {
  const dim3 g(nblk, sel_items(items));
  switch (nv) {
#define X(k) case k: k_mdot_df<k><<<g, KB, 0, s>>>(n, items, V, w, part, nblk, g_sel.list, cnt, out, outd); break;
    EHS_NV_CASES(X)
#undef X
    default: break;
  }
}
void launch_mupdate_df(long long n, int items, int nv, const float4* V, const float4* h, float4* w,
                       float4* part, int nblk, int dot, float2* nrm_part, cudaStream_t s, int* cnt, float4* out,
                       double2* outd, double* nrm, float2* inv, int store) {
  const dim3 g(nblk, sel_items(items));
  switch (nv) {
#define X(k) case k: k_mupdate_df<k><<<g, KB, 0, s>>>(n, items, V, h, w, part, nblk, dot, nrm_part, g_sel.list, \
                                                      cnt, out, outd, nrm, inv, store); break;
    EHS_NV_CASES(X)
#undef X
    default: break;
  }
}
void launch_update_scale_cast_df(long long n, int items, int nv, const float4* V, const float4* h, const float4* w,
                                 const float2* inv, float4* out, float2* out32, int nblk, cudaStream_t s,
                                 const float4* h0) {
  // no block partials here: the grid is sized for this kernel's 3 CTAs per SM (one wave per
  // item), not by the reduction kernels' nblk
  (void)nblk;
  long long gb = (n + KB - 1) / KB;
  if (gb > 3 * 152) gb = 3 * 152;
  const int nb3 = (int)(gb < 1 ? 1 : gb);
  const dim3 g(nb3, sel_items(items));
  switch (nv) {
#define X(k) case k: k_update_scale_cast_df<k><<<g, KB, 0, s>>>(n, items, V, h0, h, w, inv, out, out32, nb3, g_sel.list); \
    break;
    EHS_NV_CASES(X)
#undef X
    default: break;
  }
}
void launch_mdot2_df(long long n, int items, int j, const float4* V, const float4* w, float4* part, int nblk,
                     cudaStream_t s, int* cnt, float4* coef, double2* outd) {
  const dim3 g(2 * nblk, sel_items(items));
  switch (j + 1) {
#define X(k) case k: k_mdot2_df<k><<<g, KB, 0, s>>>(n, items, V, w, part, nblk, g_sel.list, cnt, coef, outd); break;
    EHS_NV_CASES(X)
#undef X
    default: break;
  }
}
void launch_dupdate_df(long long n, int items, int j, float4* V, const float4* w, const float4* coef,
                       float2* out32, cudaStream_t s) {
  long long gb = (n + KB - 1) / KB;   // as launch_update_scale_cast_df: 3 CTAs per SM, one wave per item
  if (gb > 3 * 152) gb = 3 * 152;
  const dim3 g((unsigned)(gb < 1 ? 1 : gb), sel_items(items));
  float4* vj = V + (size_t)j * items * n;
  float4* vn = V + (size_t)(j + 1) * items * n;
  switch (j) {
#define X(k) case k: k_dupdate_df<k><<<g, KB, 0, s>>>(n, items, V, vj, vn, w, coef, out32, g_sel.list); break;
    X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)   // j <= 10: 2 j + 3 <= KDS
#undef X
    default: break;
  }
}
void launch_scale_cast_df(long long n, int items, const float4* w, const float2* inv, float4* out, float2* out32,
                          cudaStream_t s) {
  k_scale_cast_df<<<dim3(nb(n, 256), sel_items(items)), 256, 0, s>>>(n, w, inv, out, out32, g_sel.list);
}
void launch_norm_part_df(long long n, int items, const float4* w, float2* part, int nblk, cudaStream_t s) {
  k_norm_part_df<<<dim3(nblk, sel_items(items)), KB, 0, s>>>(n, w, part, nblk, g_sel.list);
}
void launch_reduce_parts_df(int items, int nv, int nblk, const float4* part, float4* out, double2* outd,
                            cudaStream_t s) {
  const int nout = (int)sel_items(items) * nv;
  k_reduce_parts_df<<<nb((long long)nout * 32, 128), 128, 0, s>>>(nout, nblk, part, out, outd, nv, g_sel.list);
}
void launch_reduce_norm_df(int items, int nblk, const float2* part, double* out, float2* inv, cudaStream_t s) {
  const int ni = (int)sel_items(items);
  k_reduce_norm_df<<<nb((long long)ni * 32, 128), 128, 0, s>>>(ni, nblk, part, out, inv, g_sel.list);
}
void launch_scale_df(long long n, int items, const float4* w, const float2* inv, float4* out, cudaStream_t s) {
  k_scale_df<<<dim3(nb(n, 256), sel_items(items)), 256, 0, s>>>(n, w, inv, out, g_sel.list);
}
void launch_xupdate_df(long long n, int items, int m, const float2* Z, const float4* y, const int* kused,
                       float4* x, cudaStream_t s) {
  k_xupdate_df<<<dim3(nb(n, 256), items), 256, 0, s>>>(n, items, m, Z, y, kused, x);
}
void launch_d2_to_df(long long n, const double2* in, float4* out, cudaStream_t s) {
  k_d2_to_df<<<nb(n, 256), 256, 0, s>>>(n, in, out);
}
void launch_df_to_d2(long long n, const float4* in, double2* out, cudaStream_t s) {
  k_df_to_d2<<<nb(n, 256), 256, 0, s>>>(n, in, out);
}
void launch_df_to_f2(long long n, const float4* in, float2* out, cudaStream_t s) {
  k_df_to_f2<<<nb(n, 256), 256, 0, s>>>(n, in, out);
}
void launch_coef_df(long long n, const Coef4<double>* in, void* out, cudaStream_t s) {
  k_coef_df<<<nb(n, 256), 256, 0, s>>>(n, in, (Coef4df*)out);
}
void launch_apply_df_tables(const Grid& g, int nsets, const Coef4<double>* cf, double h, float4* dg, float2* vm,
                            cudaStream_t s) {
  const long long nv = (long long)(g.n[0] + 1) * (g.n[1] + 1);
  k_apply_df_tables<<<dim3((unsigned)((nv + 255) / 256), nsets), 256, 0, s>>>(g, cf, 1.0 / (h * h), dg, vm);
}
void launch_fine_apply_df(const Grid& g, int items, int nrhs, const void* cf, double h, double alpha,
                          const void* x, int x_is_c64, const float4* b, float4* y, int mode, cudaStream_t s,
                          const float4* dg, const float2* vm) {
  const FinePdf P = mkPdf(h, alpha);
  const dim3 grid(nb(g.ncell, 128), sel_items(items));
  const Coef4df* c = (const Coef4df*)cf;
  if (g.d == 2 && alpha == 0.0 && dg && vm) {   // the setup-time tables of K
    if (x_is_c64) k_fine_apply_df2t<float2><<<grid, 128, 0, s>>>(g, nrhs, c, dg, vm, P, (const float2*)x, b, y, mode,
                                                                 g_sel.list);
    else k_fine_apply_df2t<float4><<<grid, 128, 0, s>>>(g, nrhs, c, dg, vm, P, (const float4*)x, b, y, mode,
                                                        g_sel.list);
    return;
  }
  if (g.d == 2) {
    if (x_is_c64) k_fine_apply_df<float2, 2><<<grid, 128, 0, s>>>(g, nrhs, c, P, (const float2*)x, b, y, mode, g_sel.list);
    else k_fine_apply_df<float4, 2><<<grid, 128, 0, s>>>(g, nrhs, c, P, (const float4*)x, b, y, mode, g_sel.list);
  } else {
    if (x_is_c64) k_fine_apply_df<float2, 3><<<grid, 128, 0, s>>>(g, nrhs, c, P, (const float2*)x, b, y, mode, g_sel.list);
    else k_fine_apply_df<float4, 3><<<grid, 128, 0, s>>>(g, nrhs, c, P, (const float4*)x, b, y, mode, g_sel.list);
  }
}
void launch_dense_apply_df(int N, int items, int nrhs, const float4* inv, const float2* r, float2* x,
                           cudaStream_t s) {
  const int wpb = 8;
  k_dense_apply_df<<<dim3((N + wpb - 1) / wpb, sel_items(items)), 32 * wpb, 0, s>>>(N, nrhs, inv, r, x, g_sel.list);
}

}  // namespace ehs
