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

// ---------------------------------------------------------------------------------------------
// Persistent form: one cooperative launch runs a whole solve for one right-hand side.  Every phase
// works on the same 32 x 16 tiles (CTA b takes tiles b, b + G, ...), so a CTA touches only its own
// tiles' nodes and, while staging an operator tile, their halos.  The three inner-product
// reductions of an iteration are its only grid barriers:
//   op1: p_i = r + beta (p_{i-1} - omega v) formed at the staged cells (p_0 = r) and written at the
//        own nodes; v = M p_i; partial r_hat^H v                        -> reduce: alpha
//   op2: s = r - alpha v formed at the staged cells, written at the own nodes; t = M s; partials
//        t^H s and t^H t                                                -> reduce: omega
//   xr:  x += alpha p_i + omega s, r = s - omega t at the own nodes; partials r_hat^H r and
//        ||r||^2                                                        -> reduce: rho, stop, beta
// The halo values an operator phase forms come from vectors written before the last barrier, or
// from p_{i-1} and v_{i-1}, which live in the other of two alternating buffers while the owners
// write p_i and v_i.  Partials are FP64 per CTA; after a barrier every CTA adds all CTAs' partials in the
// same order, so every CTA holds the same scalars and takes the same decisions.  The update
// formulas and stop tests are those of the launch-per-step kernels above.
namespace {

constexpr int PT = 256;               // threads of the persistent kernel
constexpr int PTX = 32, PTY = 16;     // tile shape
constexpr long long kBcgSpin = 4000000000LL;  // clock budget of one barrier wait (~2 s at 2 GHz)

template <typename T>
__device__ __forceinline__ cx<T> ldcg2(const cx<T>* p);
template <>
__device__ __forceinline__ cx<float> ldcg2<float>(const cx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return mk<float>(v.x, v.y);
}
template <>
__device__ __forceinline__ cx<double> ldcg2<double>(const cx<double>* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return mk<double>(v.x, v.y);
}

__device__ __forceinline__ bool bar_failed(const hz::BicgBarrier* b) { return *((volatile const int*)&b->err) != 0; }

// Grid barrier: the last CTA to arrive bumps the generation; the others wait for it, each wait
// bounded by kBcgSpin clock cycles (then the error flag is set and every CTA returns).
__device__ __forceinline__ bool bcg_sync(hz::BicgBarrier* b, unsigned G) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&b->count, 1u) == G - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (bar_failed(b)) break;
        if (clock64() - t0 > kBcgSpin) {
          atomicExch(&b->err, 1);
          break;
        }
        __nanosleep(40);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return !bar_failed(b);
}

// CTA sum of four per-thread FP64 values, stored as this CTA's partials part[k * G + bid].
__device__ __forceinline__ void cta_partials(double (&a)[4], double* part, unsigned bid, unsigned G,
                                             double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double v = warp_sum(a[k]);
    if (lane == 0) red[wid * 4 + k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0;
    for (int w = 0; w < PT / 32; ++w) s += red[w * 4 + threadIdx.x];
    part[(size_t)threadIdx.x * G + bid] = s;
  }
}

// Barrier, then every CTA adds the G partials of each of the four values in one fixed order
// (warp k takes value k: lanes stride over the CTAs, then a shuffle tree) into out[0..3].
__device__ __forceinline__ bool bcg_reduce(hz::BicgBarrier* bar, unsigned G, const double* part, double* out) {
  if (!bcg_sync(bar, G)) return false;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < 4) {
    double s = 0;
    for (int b = lane; b < (int)G; b += 32) s += __ldcg(part + (size_t)wid * G + b);
    s = warp_sum(s);
    if (lane == 0) out[wid] = s;
  }
  __syncthreads();
  return true;
}

template <typename T>
__device__ __forceinline__ cx<T> cmulc(const double* c, cx<T> a) {  // c * a, c complex (double)
  return mk<T>(T(c[0]) * a.re - T(c[1]) * a.im, T(c[0]) * a.im + T(c[1]) * a.re);
}

// Staged value of p_i = r + beta (p_prev - omega v) (or r at the first iteration).
template <typename T>
struct PSrc {
  const cx<T>*r, *pp, *v;
  int nx;
  bool first;
  const double *beta, *omega;
  __device__ __forceinline__ cx<T> operator()(int gx, int gy) const {
    const size_t e = (size_t)gy * nx + gx;
    const cx<T> ri = ldcg2<T>(r + e);
    if (first) return ri;
    const cx<T> d = ldcg2<T>(pp + e) - cmulc<T>(omega, ldcg2<T>(v + e));
    return ri + cmulc<T>(beta, d);
  }
};

// Staged value of s = r - alpha v.
template <typename T>
struct SSrc {
  const cx<T>*r, *v;
  int nx;
  const double* alpha;
  __device__ __forceinline__ cx<T> operator()(int gx, int gy) const {
    const size_t e = (size_t)gy * nx + gx;
    return ldcg2<T>(r + e) - cmulc<T>(alpha, ldcg2<T>(v + e));
  }
};

template <typename T, int R>
__global__ void __launch_bounds__(PT) k_bicg_persist(OpP<T> P, const cx<T>* __restrict__ b, cx<T>* x, cx<T>* r,
                                                     cx<T>* p0, cx<T>* p1, cx<T>* v0, cx<T>* v1, cx<T>* s, cx<T>* t,
                                                     double* part, BicgState* st, hz::BicgBarrier* bar, int cap,
                                                     double tol) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[PT / 32 * 4];
  __shared__ double sc[4];
  const unsigned bid = blockIdx.x, G = gridDim.x;
  const int tilesx = (P.nx + PTX - 1) / PTX, tilesy = (P.ny + PTY - 1) / PTY, ntiles = tilesx * tilesy;
  const size_t n = (size_t)P.nx * P.ny;
  unsigned rc = 0;  // reductions so far: partial buffer rc & 1
  auto partbuf = [&]() { return part + (size_t)(rc & 1) * 4 * G; };
  // own nodes of this CTA's tiles: e for tile slot t and cell c (false outside the grid)
  auto own = [&](int tile, int c, size_t& e) -> bool {
    const int ox = c % PTX, oy = c / PTX;
    const int gx = (tile % tilesx) * PTX + ox, gy = (tile / tilesx) * PTY + oy;
    e = (size_t)gy * P.nx + gx;
    return gx < P.nx && gy < P.ny;
  };

  // r = b at the own nodes; ||b||^2
  {
    double a[4] = {0, 0, 0, 0};
    for (int tile = bid; tile < ntiles; tile += G)
      for (int c = threadIdx.x; c < PTX * PTY; c += PT) {
        size_t e;
        if (!own(tile, c, e)) continue;
        const cx<T> bi = b[e];
        r[e] = bi;
        a[0] += double(bi.re) * double(bi.re) + double(bi.im) * double(bi.im);
      }
    cta_partials(a, partbuf(), bid, G, red);
    if (!bcg_reduce(bar, G, partbuf(), sc)) return;
    ++rc;
  }
  const double bn2 = sc[0];
  const double tol2 = tol * tol * bn2;
  double rho[2] = {bn2, 0.0}, alpha[2] = {0, 0}, omega[2] = {0, 0}, beta[2] = {0, 0};
  double rn2 = bn2, done = bn2 > 0 ? 0.0 : 1.0;
  int its = 0;
  const TileView<T, R> tv0 = make_tile<T, R>(smem, PTX, PTY, 0, 0);
  for (; done == 0.0 && its < cap;) {
    cx<T>* pp = (its & 1) ? p0 : p1;  // p_{i-1}
    cx<T>* pn = (its & 1) ? p1 : p0;  // p_i
    cx<T>* vp = (its & 1) ? v0 : v1;  // v_{i-1}
    cx<T>* v = (its & 1) ? v1 : v0;   // v_i
    // ---- op1: p_i, v = M p_i, partial r_hat^H v
    {
      double a[4] = {0, 0, 0, 0};
      for (int tile = bid; tile < ntiles; tile += G) {
        const int ox0 = (tile % tilesx) * PTX, oy0 = (tile / tilesx) * PTY;
        TileView<T, R> tv = tv0;
        tv.ox0 = ox0;
        tv.oy0 = oy0;
        tile_fill<T, R>(tv, P, PSrc<T>{r, pp, vp, P.nx, its == 0, beta, omega});
        for (int c = threadIdx.x; c < PTX * PTY; c += PT) {
          const int ox = c % PTX, oy = c / PTX;
          const int gx = ox0 + ox, gy = oy0 + oy;
          if (gx >= P.nx || gy >= P.ny) continue;
          const size_t e = (size_t)gy * P.nx + gx;
          const cx<T> vi = tile_op<T, R>(tv, P, ox, oy);
          pn[e] = tv.u(ox + R, oy + R);
          v[e] = vi;
          const cx<T> bi = b[e];
          a[0] += double(bi.re) * double(vi.re) + double(bi.im) * double(vi.im);
          a[1] += double(bi.re) * double(vi.im) - double(bi.im) * double(vi.re);
        }
        __syncthreads();  // the tile is restaged for the next one
      }
      cta_partials(a, partbuf(), bid, G, red);
      if (!bcg_reduce(bar, G, partbuf(), sc)) return;
      ++rc;
      const double dr = sc[0], di = sc[1], d = dr * dr + di * di;
      if (!(d > 0) || !isfinite(d)) {  // breakdown: r_hat orthogonal to v
        done = 2.0;
        break;
      }
      alpha[0] = (rho[0] * dr + rho[1] * di) / d;
      alpha[1] = (rho[1] * dr - rho[0] * di) / d;
    }
    // ---- op2: s = r - alpha v, t = M s, partials t^H s and t^H t
    {
      double a[4] = {0, 0, 0, 0};
      for (int tile = bid; tile < ntiles; tile += G) {
        const int ox0 = (tile % tilesx) * PTX, oy0 = (tile / tilesx) * PTY;
        TileView<T, R> tv = tv0;
        tv.ox0 = ox0;
        tv.oy0 = oy0;
        tile_fill<T, R>(tv, P, SSrc<T>{r, v, P.nx, alpha});
        for (int c = threadIdx.x; c < PTX * PTY; c += PT) {
          const int ox = c % PTX, oy = c / PTX;
          const int gx = ox0 + ox, gy = oy0 + oy;
          if (gx >= P.nx || gy >= P.ny) continue;
          const size_t e = (size_t)gy * P.nx + gx;
          const cx<T> ti = tile_op<T, R>(tv, P, ox, oy);
          const cx<T> si = tv.u(ox + R, oy + R);
          s[e] = si;
          t[e] = ti;
          a[0] += double(ti.re) * double(si.re) + double(ti.im) * double(si.im);
          a[1] += double(ti.re) * double(si.im) - double(ti.im) * double(si.re);
          a[2] += double(ti.re) * double(ti.re) + double(ti.im) * double(ti.im);
        }
        __syncthreads();
      }
      cta_partials(a, partbuf(), bid, G, red);
      if (!bcg_reduce(bar, G, partbuf(), sc)) return;
      ++rc;
      const double ttr = sc[2];
      omega[0] = ttr > 0 ? sc[0] / ttr : 0.0;
      omega[1] = ttr > 0 ? sc[1] / ttr : 0.0;
    }
    // ---- xr: x += alpha p_i + omega s, r = s - omega t, partials r_hat^H r and ||r||^2
    {
      double a[4] = {0, 0, 0, 0};
      for (int tile = bid; tile < ntiles; tile += G)
        for (int c = threadIdx.x; c < PTX * PTY; c += PT) {
          size_t e;
          if (!own(tile, c, e)) continue;
          const cx<T> si = s[e];
          x[e] = x[e] + cmulc<T>(alpha, pn[e]) + cmulc<T>(omega, si);
          const cx<T> ri = si - cmulc<T>(omega, t[e]);
          r[e] = ri;
          const cx<T> bi = b[e];
          a[0] += double(bi.re) * double(ri.re) + double(bi.im) * double(ri.im);
          a[1] += double(bi.re) * double(ri.im) - double(bi.im) * double(ri.re);
          a[2] += double(ri.re) * double(ri.re) + double(ri.im) * double(ri.im);
        }
      cta_partials(a, partbuf(), bid, G, red);
      if (!bcg_reduce(bar, G, partbuf(), sc)) return;
      ++rc;
      const double nr = sc[0], ni = sc[1];
      rn2 = sc[2];
      ++its;
      if (!isfinite(rn2) || !isfinite(nr) || !isfinite(ni)) {
        done = 2.0;
      } else if (rn2 <= tol2) {
        done = 1.0;
      } else if ((nr == 0 && ni == 0) || (omega[0] == 0 && omega[1] == 0)) {
        done = 2.0;  // breakdown: the next direction is undefined
      } else {
        const double d1 = rho[0] * rho[0] + rho[1] * rho[1];
        const double ar = (nr * rho[0] + ni * rho[1]) / d1, ai = (ni * rho[0] - nr * rho[1]) / d1;
        const double d2 = omega[0] * omega[0] + omega[1] * omega[1];
        const double br = (alpha[0] * omega[0] + alpha[1] * omega[1]) / d2;
        const double bi = (alpha[1] * omega[0] - alpha[0] * omega[1]) / d2;
        beta[0] = ar * br - ai * bi;
        beta[1] = ar * bi + ai * br;
        rho[0] = nr;
        rho[1] = ni;
      }
    }
  }
  if (bid == 0 && threadIdx.x == 0) {
    BicgState o = *st;
    o.rho[0] = rho[0];
    o.rho[1] = rho[1];
    o.alpha[0] = alpha[0];
    o.alpha[1] = alpha[1];
    o.omega[0] = omega[0];
    o.omega[1] = omega[1];
    o.beta[0] = beta[0];
    o.beta[1] = beta[1];
    o.bn2 = bn2;
    o.rn2 = rn2;
    o.tol2 = tol2;
    o.done = done;
    o.its = its;
    o.total_its += its;
    if (!isfinite(rn2)) o.nonfinite += 1.0;
    *st = o;
  }
  (void)n;
}

template <typename T, int R>
size_t bicg_smem() {
  return tile_smem_bytes<T, R>(PTX, PTY);
}

template <typename T, int R>
int bicg_grid_t(int nx, int ny) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  const size_t sm = bicg_smem<T, R>();
  if (hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_bicg_persist<T, R>), sm) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bicg_persist<T, R>, PT, sm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const long long tiles = (long long)((nx + PTX - 1) / PTX) * ((ny + PTY - 1) / PTY);
  const long long most = (long long)per * sms;
  return (int)std::min<long long>(tiles, std::min<long long>(most, 2LL * sms));
}

template <typename T, int R>
cudaError_t bicg_persist_t(hz::Ctx& c, const hz::OpDesc& d, const void* b, void* x, void* work, double* part,
                           BicgState* st, hz::BicgBarrier* bar, int cap, double tol, int grid) {
  OpP<T> P;
  P.nx = d.nx;
  P.ny = d.ny;
  P.R = d.R;
  P.bc = d.bc;
  P.srow = d.srow;
  P.c = T(d.c);
  P.H = T(d.H);
  P.ks = T(d.ks);
  P.sr = T(d.sr);
  P.si = T(d.si);
  P.ksr = T(d.ks * d.sr);
  P.ksi = T(d.ks * d.si);
  for (int i = 0; i < 7; ++i) {
    P.m[i] = T(d.m[i]);
    P.l[i] = T(d.l[i]);
  }
  if constexpr (sizeof(T) == 8) P.k = reinterpret_cast<const T*>(d.k_d);
  else P.k = reinterpret_cast<const T*>(d.k_f);
  P.kstride = 0;
  const size_t n = d.n();
  const cx<T>* bb = reinterpret_cast<const cx<T>*>(b);
  cx<T>* xx = reinterpret_cast<cx<T>*>(x);
  cx<T>* w = reinterpret_cast<cx<T>*>(work);
  cx<T>*r = w, *p0 = w + n, *p1 = w + 2 * n, *v0 = w + 3 * n, *v1 = w + 4 * n, *s = w + 5 * n, *t = w + 6 * n;
  const size_t sm = bicg_smem<T, R>();
  cudaError_t e = hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_bicg_persist<T, R>), sm);
  if (e != cudaSuccess) return e;
  void* args[] = {&P, &bb, &xx, &r, &p0, &p1, &v0, &v1, &s, &t, &part, &st, &bar, &cap, &tol};
  hz::ProfScope ps(c, hz::F_BICG, 0.0);
  return cudaLaunchCooperativeKernel((const void*)k_bicg_persist<T, R>, dim3(grid), dim3(PT), args, sm, c.s);
}

}  // namespace

namespace hz {

int bicg_persist_grid(int dt, int R, int nx, int ny) {
  if (dt == C128) {
    if (R == 1) return bicg_grid_t<double, 1>(nx, ny);
    if (R == 2) return bicg_grid_t<double, 2>(nx, ny);
    if (R == 3) return bicg_grid_t<double, 3>(nx, ny);
  } else {
    if (R == 1) return bicg_grid_t<float, 1>(nx, ny);
    if (R == 2) return bicg_grid_t<float, 2>(nx, ny);
    if (R == 3) return bicg_grid_t<float, 3>(nx, ny);
  }
  return 0;
}

cudaError_t launch_bicg_persist(Ctx& c, const OpDesc& M, int dt, const void* b, void* x, void* work, double* part,
                                BicgState* st, BicgBarrier* bar, int cap, double tol, int grid) {
#define HZ_BP(T_, R_) return bicg_persist_t<T_, R_>(c, M, b, x, work, part, st, bar, cap, tol, grid)
  if (grid < 1) return cudaErrorInvalidValue;
  if (dt == C128) {
    if (M.R == 1) HZ_BP(double, 1);
    if (M.R == 2) HZ_BP(double, 2);
    if (M.R == 3) HZ_BP(double, 3);
  } else {
    if (M.R == 1) HZ_BP(float, 1);
    if (M.R == 2) HZ_BP(float, 2);
    if (M.R == 3) HZ_BP(float, 3);
  }
#undef HZ_BP
  return cudaErrorInvalidValue;
}

}  // namespace hz
