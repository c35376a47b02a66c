// Bi-CGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput. 13(2), 1992) for the CSLP inverse on
// the levels beyond the multigrid ones: the Krylov solver of the earlier multilevel work
// (Section 3.2) and of the tolerance study of Section 4.1, offered beside GMRES.
//
// One iteration, zero initial guess, shadow residual r_hat = b:
//   p = r + beta (p - omega v)     beta = (rho / rho_old)(alpha / omega), p = r first
//   v = M p,  alpha = rho / (r_hat^H v),  s = r - alpha v
//   t = M s,  omega = t^H s / t^H t
//   x += alpha p + omega s,  r = s - omega t,  rho = r_hat^H r,  stop when ||r|| <= tol ||b||
// The operator applies are the level-operator kernels; this file holds the fused vector
// updates, the inner products and the scalar steps.  Scalars live in device memory (one
// BicgState per right-hand side), so no iteration waits for the host; a right-hand side that
// has stopped makes every later update kernel return early for it.  Inner products are
// deterministic: each CTA writes its partial sums, the scalar kernel adds them in a fixed order.
#include "hz_device.cuh"
#include "hz_internal.h"

using namespace hzd;
using hz::BicgState;

namespace {

constexpr int NT = 256;
constexpr int MAXP = 152 * 4;  // CTAs per right-hand side in the reduction passes
constexpr int NPAIR = 2;       // inner products per pass
constexpr int PSTRIDE = 2 * NPAIR;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-sum the NPAIR complex accumulators and store them as this CTA's partials.
__device__ __forceinline__ void store_partials(double (&acc)[PSTRIDE], double* __restrict__ part) {
  __shared__ double red[NT / 32][PSTRIDE];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < PSTRIDE; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < PSTRIDE) {
    double s = 0;
    for (int w = 0; w < NT / 32; ++w) s += red[w][threadIdx.x];
    part[threadIdx.x] = s;
  }
}

template <typename T>
__device__ __forceinline__ void acc_dot(double (&acc)[PSTRIDE], int k, cx<T> a, cx<T> b) {
  // conj(a) * b
  acc[2 * k] += double(a.re) * double(b.re) + double(a.im) * double(b.im);
  acc[2 * k + 1] += double(a.re) * double(b.im) - double(a.im) * double(b.re);
}

// partials of a0^H b0 and (npair == 2) a1^H b1, per right-hand side blockIdx.y
template <typename T>
__global__ void __launch_bounds__(NT) k_bcg_dots(const cx<T>* __restrict__ a0, const cx<T>* __restrict__ b0,
                                                 const cx<T>* __restrict__ a1, const cx<T>* __restrict__ b1,
                                                 int npair, size_t n, double* __restrict__ part,
                                                 const BicgState* __restrict__ st) {
  const int q = blockIdx.y;
  if (st && st[q].done != 0.0) return;
  const size_t off = (size_t)q * n;
  double acc[PSTRIDE] = {};
  for (size_t i = (size_t)blockIdx.x * NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
    acc_dot<T>(acc, 0, a0[off + i], b0[off + i]);
    if (npair == 2) acc_dot<T>(acc, 1, a1[off + i], b1[off + i]);
  }
  store_partials(acc, part + ((size_t)q * gridDim.x + blockIdx.x) * PSTRIDE);
}

// sum of the P partials of pair k for right-hand side q, in CTA order
__device__ __forceinline__ void sum_parts(const double* __restrict__ part, int q, int P, int k, double& re,
                                          double& im) {
  re = 0;
  im = 0;
  const double* p = part + (size_t)q * P * PSTRIDE;
  for (int b = 0; b < P; ++b) {
    re += p[(size_t)b * PSTRIDE + 2 * k];
    im += p[(size_t)b * PSTRIDE + 2 * k + 1];
  }
}

// step 0: from ||b||^2 set rho = ||b||^2 (r = r_hat = b), beta = omega = 0 (so p = r), stop at b = 0
__global__ void k_bcg_start(const double* __restrict__ part, int P, int nb, double tol, BicgState* __restrict__ st) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nb) return;
  double re, im;
  sum_parts(part, q, P, 0, re, im);
  BicgState s = {};
  s.bn2 = re;
  s.rn2 = re;
  s.tol2 = tol * tol * re;
  s.rho[0] = re;
  s.done = re > 0 ? 0.0 : 1.0;
  st[q] = s;
}

// alpha = rho / (r_hat^H v)
__global__ void k_bcg_alpha(const double* __restrict__ part, int P, int nb, BicgState* __restrict__ st) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nb || st[q].done != 0.0) return;
  double dr, di;
  sum_parts(part, q, P, 0, dr, di);
  const double d = dr * dr + di * di;
  if (!(d > 0) || !isfinite(d)) {
    st[q].done = 2.0;  // breakdown: r_hat orthogonal to v
    return;
  }
  const double rr = st[q].rho[0], ri = st[q].rho[1];
  st[q].alpha[0] = (rr * dr + ri * di) / d;
  st[q].alpha[1] = (ri * dr - rr * di) / d;
}

// omega = t^H s / t^H t  (pair 0: t^H s, pair 1: t^H t); t = 0 means s = 0: omega = 0
__global__ void k_bcg_omega(const double* __restrict__ part, int P, int nb, BicgState* __restrict__ st) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nb || st[q].done != 0.0) return;
  double tsr, tsi, ttr, tti;
  sum_parts(part, q, P, 0, tsr, tsi);
  sum_parts(part, q, P, 1, ttr, tti);
  st[q].omega[0] = ttr > 0 ? tsr / ttr : 0.0;
  st[q].omega[1] = ttr > 0 ? tsi / ttr : 0.0;
}

// after x, r: rho_new = r_hat^H r (pair 0), ||r||^2 (pair 1); stop or form beta
__global__ void k_bcg_rho(const double* __restrict__ part, int P, int nb, BicgState* __restrict__ st) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nb || st[q].done != 0.0) return;
  BicgState s = st[q];
  double nr, ni, rn2, dummy;
  sum_parts(part, q, P, 0, nr, ni);
  sum_parts(part, q, P, 1, rn2, dummy);
  s.its += 1.0;
  s.rn2 = rn2;
  if (!isfinite(rn2) || !isfinite(nr) || !isfinite(ni)) {
    s.done = 2.0;
  } else if (rn2 <= s.tol2) {
    s.done = 1.0;
  } else if ((nr == 0 && ni == 0) || (s.omega[0] == 0 && s.omega[1] == 0)) {
    s.done = 2.0;  // breakdown: the next direction is undefined
  } else {
    // beta = (rho_new / rho) * (alpha / omega)
    const double d1 = s.rho[0] * s.rho[0] + s.rho[1] * s.rho[1];
    const double ar = (nr * s.rho[0] + ni * s.rho[1]) / d1, ai = (ni * s.rho[0] - nr * s.rho[1]) / d1;
    const double d2 = s.omega[0] * s.omega[0] + s.omega[1] * s.omega[1];
    const double br = (s.alpha[0] * s.omega[0] + s.alpha[1] * s.omega[1]) / d2;
    const double bi = (s.alpha[1] * s.omega[0] - s.alpha[0] * s.omega[1]) / d2;
    s.beta[0] = ar * br - ai * bi;
    s.beta[1] = ar * bi + ai * br;
    s.rho[0] = nr;
    s.rho[1] = ni;
  }
  st[q] = s;
}

template <typename T>
__device__ __forceinline__ cx<T> cscale(const double* c, cx<T> a) {
  return mk<T>(T(c[0]) * a.re - T(c[1]) * a.im, T(c[0]) * a.im + T(c[1]) * a.re);
}

// p = r + beta (p - omega v)
template <typename T>
__global__ void __launch_bounds__(NT) k_bcg_p(const cx<T>* __restrict__ r, cx<T>* __restrict__ p,
                                              const cx<T>* __restrict__ v, size_t n,
                                              const BicgState* __restrict__ st) {
  const int q = blockIdx.y;
  if (st[q].done != 0.0) return;
  const double* beta = st[q].beta;
  const double* omega = st[q].omega;
  const size_t off = (size_t)q * n;
  for (size_t i = (size_t)blockIdx.x * NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
    const cx<T> d = p[off + i] - cscale<T>(omega, v[off + i]);
    p[off + i] = r[off + i] + cscale<T>(beta, d);
  }
}

// s = r - alpha v
template <typename T>
__global__ void __launch_bounds__(NT) k_bcg_s(const cx<T>* __restrict__ r, const cx<T>* __restrict__ v,
                                              cx<T>* __restrict__ s, size_t n, const BicgState* __restrict__ st) {
  const int q = blockIdx.y;
  if (st[q].done != 0.0) return;
  const double* alpha = st[q].alpha;
  const size_t off = (size_t)q * n;
  for (size_t i = (size_t)blockIdx.x * NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT)
    s[off + i] = r[off + i] - cscale<T>(alpha, v[off + i]);
}

// x += alpha p + omega s, r = s - omega t, with the partials of r_hat^H r and ||r||^2
template <typename T>
__global__ void __launch_bounds__(NT) k_bcg_xr(cx<T>* __restrict__ x, const cx<T>* __restrict__ p,
                                               const cx<T>* __restrict__ s, const cx<T>* __restrict__ t,
                                               cx<T>* __restrict__ r, const cx<T>* __restrict__ rhat, size_t n,
                                               double* __restrict__ part, const BicgState* __restrict__ st) {
  const int q = blockIdx.y;
  if (st[q].done != 0.0) return;
  const double* alpha = st[q].alpha;
  const double* omega = st[q].omega;
  const size_t off = (size_t)q * n;
  double acc[PSTRIDE] = {};
  for (size_t i = (size_t)blockIdx.x * NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
    const cx<T> si = s[off + i];
    x[off + i] = x[off + i] + cscale<T>(alpha, p[off + i]) + cscale<T>(omega, si);
    const cx<T> ri = si - cscale<T>(omega, t[off + i]);
    r[off + i] = ri;
    acc_dot<T>(acc, 0, rhat[off + i], ri);
    acc_dot<T>(acc, 1, ri, ri);
  }
  store_partials(acc, part + ((size_t)q * gridDim.x + blockIdx.x) * PSTRIDE);
}

inline unsigned scal_grid(int nb) { return (unsigned)((nb + 127) / 128); }

template <typename T>
const cx<T>* C(const void* p) {
  return reinterpret_cast<const cx<T>*>(p);
}
template <typename T>
cx<T>* W(void* p) {
  return reinterpret_cast<cx<T>*>(p);
}

}  // namespace

namespace hz {

int bicg_parts(size_t n) {
  size_t b = (n + NT * 4 - 1) / (NT * 4);
  if (b > (size_t)MAXP) b = MAXP;
  return (int)(b > 0 ? b : 1);
}

size_t bicg_part_bytes(size_t n, int nb) { return sizeof(double) * PSTRIDE * (size_t)bicg_parts(n) * nb; }

cudaError_t launch_bicg_start(Ctx& c, int dt, const void* b, size_t n, int nb, double tol, double* part,
                              BicgState* st) {
  const int P = bicg_parts(n);
  {
    ProfScope ps(c, F_DOT, (double)nb * n * elem_bytes(dt));
    dim3 grid(P, nb);
    if (dt == C128)
      k_bcg_dots<double><<<grid, NT, 0, c.s>>>(C<double>(b), C<double>(b), nullptr, nullptr, 1, n, part, nullptr);
    else
      k_bcg_dots<float><<<grid, NT, 0, c.s>>>(C<float>(b), C<float>(b), nullptr, nullptr, 1, n, part, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  ProfScope ps(c, F_REDUCE, 0.0);
  k_bcg_start<<<scal_grid(nb), 128, 0, c.s>>>(part, P, nb, tol, st);
  return cudaGetLastError();
}

// which: 0 alpha from (r_hat, v); 1 omega from (t, s), (t, t)
cudaError_t launch_bicg_dots(Ctx& c, int dt, int which, const void* a0, const void* b0, const void* a1,
                             const void* b1, size_t n, int nb, double* part, BicgState* st) {
  const int P = bicg_parts(n);
  const int npair = which == 0 ? 1 : 2;
  {
    ProfScope ps(c, F_DOT, (double)nb * n * elem_bytes(dt) * (npair == 1 ? 2 : 3));
    dim3 grid(P, nb);
    if (dt == C128)
      k_bcg_dots<double><<<grid, NT, 0, c.s>>>(C<double>(a0), C<double>(b0), C<double>(a1), C<double>(b1), npair,
                                               n, part, st);
    else
      k_bcg_dots<float><<<grid, NT, 0, c.s>>>(C<float>(a0), C<float>(b0), C<float>(a1), C<float>(b1), npair, n,
                                              part, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  ProfScope ps(c, F_REDUCE, 0.0);
  if (which == 0)
    k_bcg_alpha<<<scal_grid(nb), 128, 0, c.s>>>(part, P, nb, st);
  else
    k_bcg_omega<<<scal_grid(nb), 128, 0, c.s>>>(part, P, nb, st);
  return cudaGetLastError();
}

cudaError_t launch_bicg_p(Ctx& c, int dt, const void* r, void* p, const void* v, size_t n, int nb,
                          const BicgState* st) {
  ProfScope ps(c, F_AXPY, (double)nb * n * elem_bytes(dt) * 4);
  dim3 grid(bicg_parts(n), nb);
  if (dt == C128)
    k_bcg_p<double><<<grid, NT, 0, c.s>>>(C<double>(r), W<double>(p), C<double>(v), n, st);
  else
    k_bcg_p<float><<<grid, NT, 0, c.s>>>(C<float>(r), W<float>(p), C<float>(v), n, st);
  return cudaGetLastError();
}

cudaError_t launch_bicg_s(Ctx& c, int dt, const void* r, const void* v, void* s, size_t n, int nb,
                          const BicgState* st) {
  ProfScope ps(c, F_AXPY, (double)nb * n * elem_bytes(dt) * 3);
  dim3 grid(bicg_parts(n), nb);
  if (dt == C128)
    k_bcg_s<double><<<grid, NT, 0, c.s>>>(C<double>(r), C<double>(v), W<double>(s), n, st);
  else
    k_bcg_s<float><<<grid, NT, 0, c.s>>>(C<float>(r), C<float>(v), W<float>(s), n, st);
  return cudaGetLastError();
}

cudaError_t launch_bicg_xr(Ctx& c, int dt, void* x, const void* p, const void* s, const void* t, void* r,
                           const void* rhat, size_t n, int nb, double* part, BicgState* st) {
  const int P = bicg_parts(n);
  {
    ProfScope ps(c, F_AXPY, (double)nb * n * elem_bytes(dt) * 7);
    dim3 grid(P, nb);
    if (dt == C128)
      k_bcg_xr<double><<<grid, NT, 0, c.s>>>(W<double>(x), C<double>(p), C<double>(s), C<double>(t), W<double>(r),
                                             C<double>(rhat), n, part, st);
    else
      k_bcg_xr<float><<<grid, NT, 0, c.s>>>(W<float>(x), C<float>(p), C<float>(s), C<float>(t), W<float>(r),
                                            C<float>(rhat), n, part, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  ProfScope ps(c, F_REDUCE, 0.0);
  k_bcg_rho<<<scal_grid(nb), 128, 0, c.s>>>(part, P, nb, st);
  return cudaGetLastError();
}

}  // namespace hz
