// Adjoint-state gradient of the mixed elastic Helmholtz system with respect
// to the cell-centred medium (lambda, mu, rho):
//     g_m(c) = -Re( w^H (dK/dm_c) x ),  summed over the right-hand sides of a medium,
// where x solves K x = q and w solves K^H w = e (the misfit's derivative).
// The derivative of K follows its assembly (Sec. 2.1 eq. elasticHelmSystem,
// eq. elasticHelmMass; Sec. 3 eq. elasticHelmReformulatedSystem):
//  * pressure block -1/(lambda+mu): d/dlambda = d/dmu = 1/(lambda+mu)^2;
//  * weighted Laplacian: the normal difference of u_k across cell c carries
//    mu_c; a tangential edge difference carries the mean of the 4 cells around
//    the edge (clamped), so cell c receives 1/4 per appearance;
//  * face mass -omega^2 A_f(rho (1 - i gamma/omega)): each face of cell c
//    receives -omega^2 (1 - i gamma_c/omega) / 2.
// FP64 throughout: it runs once per inversion step, not inside the solve.
#include "kernels.h"

namespace ehs {
namespace {

__device__ __forceinline__ double2 ld(const double2* p, long long i, bool ok) {
  return ok ? p[i] : make_double2(0, 0);
}
__device__ __forceinline__ double re_cmul(double2 w, double2 x) {   // Re(conj(w) x)
  return w.x * x.x + w.y * x.y;
}

template <int D>
__global__ void k_gradient(Grid g, int nrhs, const Coef4<double>* __restrict__ cf,
                           const double* __restrict__ rho, const double* __restrict__ omegas, double h,
                           const double2* __restrict__ x, const double2* __restrict__ w,
                           double* __restrict__ gl, double* __restrict__ gm, double* __restrict__ gr) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int m = blockIdx.y;
  const long long N = g.ncell;
  const Coef4<double> cc = cf[(long long)m * N + c];
  const double rc = rho[(long long)m * N + c];
  const double om = omegas[m];
  // d(-omega^2 rho (1 - i gamma/omega))/d rho = -(omega^2 - i mi/rho), half per face
  const double2 mfac = make_double2(-0.5 * om * om, 0.5 * cc.mi / rc);
  const double h2 = 1.0 / (h * h);
  int i[3];
  cell_coords(g, c, i);
  double sl = 0.0, sm = 0.0, sr = 0.0;
  for (int r = 0; r < nrhs; ++r) {
    const long long vo = ((long long)m * nrhs + r) * (D + 1) * N;
    const double2* xv = x + vo;
    const double2* wv = w + vo;
    // pressure block
    const double tp = -re_cmul(wv[(long long)D * N + c], xv[(long long)D * N + c]) * cc.kap * cc.kap;
    sl += tp;
    sm += tp;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const long long sk = stride_of(g, k);
      const double2* xk = xv + (long long)k * N;
      const double2* wk = wv + (long long)k * N;
      const bool lo_ok = i[k] >= 1, hi_ok = i[k] + 1 < g.n[k];
      const double2 xl = ld(xk, c, lo_ok), xh = ld(xk, c + sk, hi_ok);
      const double2 wl = ld(wk, c, lo_ok), wh = ld(wk, c + sk, hi_ok);
      // mass on the two faces of cell c
      const double2 s = make_double2(re_cmul(wl, xl) + re_cmul(wh, xh),
                                     (wl.x * xl.y - wl.y * xl.x) + (wh.x * xh.y - wh.y * xh.x));
      sr += -(s.x * mfac.x - s.y * mfac.y);
      // normal difference across cell c, weight mu_c
      const double2 dx = make_double2(xh.x - xl.x, xh.y - xl.y);
      const double2 dw = make_double2(wh.x - wl.x, wh.y - wl.y);
      sm += -re_cmul(dw, dx) * h2;
      // tangential edges of the two faces of cell c
#pragma unroll
      for (int j = 0; j < D; ++j) {
        if (j == k) continue;
        const long long sj = stride_of(g, j);
        for (int side = 0; side < 2; ++side) {
          const bool fok = side ? hi_ok : lo_ok;
          if (!fok) continue;
          const long long f = c + (side ? sk : 0);       // slot of the face in row i_j
          for (int e = i[j]; e <= i[j] + 1; ++e) {       // edge between rows e-1 and e
            const int c0 = max(e - 1, 0), c1 = min(e, g.n[j] - 1);
            const int mult = (c0 == i[j]) + (c1 == i[j]);
            if (!mult) continue;
            const bool up_ok = e <= g.n[j] - 1, dn_ok = e - 1 >= 0;
            const long long fu = f + (long long)(e - i[j]) * sj, fd = fu - sj;
            const double2 xu = ld(xk, fu, up_ok), xd = ld(xk, fd, dn_ok);
            const double2 wu = ld(wk, fu, up_ok), wd = ld(wk, fd, dn_ok);
            const double2 ex = make_double2(xu.x - xd.x, xu.y - xd.y);
            const double2 ew = make_double2(wu.x - wd.x, wu.y - wd.y);
            sm += -re_cmul(ew, ex) * h2 * 0.25 * mult;
          }
        }
      }
    }
  }
  gl[(long long)m * N + c] = sl;
  gm[(long long)m * N + c] = sm;
  gr[(long long)m * N + c] = sr;
}

}  // namespace

void launch_gradient(const Grid& g, int nsets, int nrhs, const Coef4<double>* cf, const double* rho,
                     const double* omegas, double h, const double2* x, const double2* w, double* gl,
                     double* gm, double* gr, cudaStream_t s) {
  const dim3 grid((unsigned)((g.ncell + 127) / 128), nsets);
  if (g.d == 2) k_gradient<2><<<grid, 128, 0, s>>>(g, nrhs, cf, rho, omegas, h, x, w, gl, gm, gr);
  else k_gradient<3><<<grid, 128, 0, s>>>(g, nrhs, cf, rho, omegas, h, x, w, gl, gm, gr);
}

}  // namespace ehs
