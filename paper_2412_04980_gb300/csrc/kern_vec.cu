// Krylov vector kernels (Algorithm 1 lines 16-23: inner products, Gram-Schmidt updates,
// norms, the final combination u = u0 + X y) and the dense multigrid coarsest solve.
//
// Reductions are deterministic: each CTA writes one partial per coefficient, a second
// kernel sums the partials in a fixed order.  FP32 vectors accumulate per thread in FP32
// and reduce across threads in FP64; FP64 vectors use FP64 throughout.
#include <type_traits>

#include <algorithm>

#include "hz_device.cuh"
#include "hz_internal.h"

using namespace hzd;

namespace {

constexpr int NT = 256;        // threads per CTA
constexpr int CV = 8;          // vectors per multi-dot CTA
constexpr int MAXP = 1216;     // element CTAs (8 per SM)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp transpose-reduction of CNT values held by every lane (CNT a power of two <= 32):
// after it, lane l (l < CNT) holds the warp sum of value (l % CNT).  Each halving step
// exchanges half of the remaining values, so a lane performs CNT - 1 + log2(32/CNT) adds
// instead of 5 * CNT for independent butterfly sums.
template <typename T, int CNT>
__device__ __forceinline__ T warp_transpose_sum(T (&v)[CNT]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int half = CNT / 2; half >= 1; half >>= 1) {
    const bool upper = (lane & half) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      T send = upper ? v[i] : v[i + half];
      T keep = upper ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  T x = v[0];
#pragma unroll
  for (int o = CNT; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;  // lane l holds the sum of value index (l & (CNT-1)) -- after the transposition
}

// Which original value index ends up in lane slot q after warp_transpose_sum<CNT>.
template <int CNT>
__device__ __forceinline__ int slot_value(int q) {
  // at each halving step with width `half`, lanes with (lane & half) keep the upper half;
  // the kept index is v[i + half] for those lanes, so bit `half` of the lane selects it.
  int idx = 0;
  for (int half = CNT / 2; half >= 1; half >>= 1)
    if (q & half) idx += half;
  return idx;
}

inline int nparts(size_t n) {
  size_t b = (n + NT * 4 - 1) / (NT * 4);
  if (b > MAXP) b = MAXP;
  return (int)(b > 0 ? b : 1);
}

// partial[by * ldp + 2*i + {0,1}] for vectors i of chunk blockIdx.x
template <typename T>
__global__ void __launch_bounds__(NT) k_multidot(const cx<T>* __restrict__ V, size_t ldv, int nv,
                                                 const cx<T>* __restrict__ w, size_t n, double* __restrict__ part,
                                                 int ldp, int with_norm, const double* __restrict__ skip) {
  __shared__ double sm[8 * 2 * CV];
  __shared__ double snorm[NT / 32];
  if (skip && skip[blockIdx.z] != 0.0) return;
  const int c0 = blockIdx.x * CV;
  const bool do_norm = with_norm && blockIdx.x == 0;
  V += (size_t)blockIdx.z * n;
  w += (size_t)blockIdx.z * n;
  part += (size_t)blockIdx.z * gridDim.y * ldp;
  const int cnt = min(CV, nv - c0);
  T ar[CV], ai[CV];
  T wn = T(0);
#pragma unroll
  for (int i = 0; i < CV; ++i) ar[i] = ai[i] = T(0);
  for (size_t e = blockIdx.y * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.y * NT) {
    cx<T> we = w[e];
    if (do_norm) wn += we.re * we.re + we.im * we.im;
#pragma unroll
    for (int i = 0; i < CV; ++i) {
      if (i < cnt) {
        cx<T> v = V[(size_t)(c0 + i) * ldv + e];
        ar[i] += v.re * we.re + v.im * we.im;
        ai[i] += v.re * we.im - v.im * we.re;
      }
    }
  }
  T vals[2 * CV];
#pragma unroll
  for (int i = 0; i < CV; ++i) {
    vals[2 * i] = ar[i];
    vals[2 * i + 1] = ai[i];
  }
  // value index held by this lane after the transposition: bit-reversed halving order
  const T ws = warp_transpose_sum<T, 2 * CV>(vals);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane < 2 * CV) sm[wid * 2 * CV + lane] = double(ws);
  if (do_norm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wn += __shfl_xor_sync(0xffffffffu, wn, o);
    if (lane == 0) snorm[wid] = double(wn);
  }
  __syncthreads();
  if (do_norm && threadIdx.x == 0) {
    double t = 0;
    for (int w2 = 0; w2 < NT / 32; ++w2) t += snorm[w2];
    part[(size_t)blockIdx.y * ldp + 2 * nv] = t;
  }
  if (threadIdx.x < 2 * CV) {
    const int q = threadIdx.x;          // slot; its value index is slot_value(q)
    double t = 0;
    for (int w = 0; w < NT / 32; ++w) t += sm[w * 2 * CV + q];
    const int vi = slot_value<2 * CV>(q);
    if ((vi >> 1) < cnt) part[(size_t)blockIdx.y * ldp + 2 * c0 + vi] = t;
  }
}

// out[j] = sum_b part[b * ldp + j], j < m (fixed order)
__global__ void __launch_bounds__(NT) k_reduce(const double* __restrict__ part, int nb, int ldp, int m,
                                               double* __restrict__ out) {
  __shared__ double sm[8];
  const int j = blockIdx.x;
  part += (size_t)blockIdx.y * nb * ldp;
  out += (size_t)blockIdx.y * m;
  if (j >= m) return;
  double s = 0;
  for (int b = threadIdx.x; b < nb; b += NT) s += part[(size_t)b * ldp + j];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < NT / 32; ++w) t += sm[w];
    out[j] = t;
  }
}

// w -= sum_i coef_i V_i ; optional partial norms of the new w
template <typename TV, typename TW>
__global__ void __launch_bounds__(NT) k_update(const cx<TV>* __restrict__ V, size_t ldv, int nv,
                                               const double* __restrict__ coef, int ldc, cx<TW>* __restrict__ w,
                                               size_t n, double* __restrict__ part, const double* __restrict__ skip) {
  extern __shared__ double scoef[];  // 2 * nv
  __shared__ double sm[8];
  if (skip && skip[blockIdx.y] != 0.0) return;
  V += (size_t)blockIdx.y * n;
  w += (size_t)blockIdx.y * n;
  coef += (size_t)blockIdx.y * ldc;
  if (part) part += (size_t)blockIdx.y * gridDim.x;
  using T = typename std::conditional<(sizeof(TW) > sizeof(TV)), TW, TV>::type;
  T* sc = reinterpret_cast<T*>(scoef);  // coefficients converted once to the arithmetic type
  for (int i = threadIdx.x; i < 2 * nv; i += NT) sc[i] = T(coef[i]);
  __syncthreads();
  T acc = T(0);
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.x * NT) {
    cx<T> x = cvt<T>(w[e]);
    for (int i = 0; i < nv; ++i) {
      cx<T> v = cvt<T>(V[(size_t)i * ldv + e]);
      T cr = sc[2 * i], ci = sc[2 * i + 1];
      x.re -= cr * v.re - ci * v.im;
      x.im -= cr * v.im + ci * v.re;
    }
    w[e] = cvt<TW>(x);
    if (part) acc += x.re * x.re + x.im * x.im;
  }
  if (part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    double s = double(acc);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int q = 0; q < NT / 32; ++q) t += sm[q];
      part[blockIdx.x] = t;
    }
  }
}

// flag[b] = 1 (skip the second Gram-Schmidt pass) when ||w'||^2 >= eta2 ||w||^2
__global__ void k_dgks(const double* __restrict__ wn, int ldw, const double* __restrict__ n1, double* __restrict__ flag,
                       int nb, double eta2) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) flag[b] = (n1[b] >= eta2 * wn[(size_t)b * ldw]) ? 1.0 : 0.0;
}

// One-iteration FGMRES cycle as a minimal-residual step (Algorithm 1 with m = 1): with v = b / ||b||,
// x = P v, w1 = A x, the least-squares coefficient is y = ||b|| conj(h11) / (|h11|^2 + h21^2) with
// h11 = v^H w1 and |h11|^2 + h21^2 = ||w1||^2, so the cycle's result y P v equals
// (w^H b / w^H w) P b with w = A P b.  d holds b^H w and ||w||^2 per right-hand side (stride 3).
__global__ void k_m1_mr(const double* __restrict__ d, int nb, double* __restrict__ coef, int* __restrict__ its,
                        int* __restrict__ calls, int* __restrict__ err) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const double hr = d[3 * b], hi = d[3 * b + 1], nw = d[3 * b + 2];
  coef[2 * b] = 0.0;
  coef[2 * b + 1] = 0.0;
  if (!isfinite(hr) || !isfinite(hi) || !isfinite(nw)) {
    atomicExch(err, 1);
    return;
  }
  if (!(nw > 0)) return;  // b = 0 (or A P b = 0): nothing to add
  coef[2 * b] = hr / nw;    // conj(b^H w) / ||w||^2
  coef[2 * b + 1] = -hi / nw;
  its[b] += 1;
  calls[b] += 1;
}

// y = D x: boundary edges times 1/2, corners times 1/4 (the symmetric scaling of the Sommerfeld
// rows), complex FP64, nb vectors of nx * ny.
__global__ void __launch_bounds__(256) k_row_scale(const cx<double>* __restrict__ x, cx<double>* __restrict__ y,
                                                   int nx, int ny) {
  const size_t n = (size_t)nx * ny, off = (size_t)blockIdx.y * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int gy = (int)(i / nx), gx = (int)(i - (size_t)gy * nx);
    const int g = (gx == 0) + (gx == nx - 1) + (gy == 0) + (gy == ny - 1);
    const double s = g == 0 ? 1.0 : (g == 1 ? 0.5 : 0.25);
    y[off + i] = s * x[off + i];
  }
}

// u += sum_i coef_i X_i
template <typename TX, typename TU>
__global__ void __launch_bounds__(NT) k_combine(const cx<TX>* __restrict__ X, size_t ldx, int nv,
                                                const double* __restrict__ coef, cx<TU>* __restrict__ u, size_t n) {
  extern __shared__ double scoef[];
  X += (size_t)blockIdx.y * n;
  u += (size_t)blockIdx.y * n;
  coef += (size_t)blockIdx.y * 2 * nv;
  using T = typename std::conditional<(sizeof(TU) > sizeof(TX)), TU, TX>::type;
  T* sc = reinterpret_cast<T*>(scoef);
  for (int i = threadIdx.x; i < 2 * nv; i += NT) sc[i] = T(coef[i]);
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.x * NT) {
    cx<T> x = cvt<T>(u[e]);
    for (int i = 0; i < nv; ++i) {
      cx<T> v = cvt<T>(X[(size_t)i * ldx + e]);
      T cr = sc[2 * i], ci = sc[2 * i + 1];
      x.re += cr * v.re - ci * v.im;
      x.im += cr * v.im + ci * v.re;
    }
    u[e] = cvt<TU>(x);
  }
}

// y = alpha * x, alpha = coef (complex) or 1/sqrt(nrm2) (recip)
template <typename T>
__global__ void __launch_bounds__(NT) k_scale(const cx<T>* __restrict__ x, cx<T>* __restrict__ y,
                                              const double* __restrict__ alpha, int recip, size_t n) {
  x += (size_t)blockIdx.y * n;
  y += (size_t)blockIdx.y * n;
  alpha += (size_t)blockIdx.y * (recip ? 1 : 2);
  double ar, ai;
  if (recip) {
    double s = alpha[0];
    ar = s > 0 ? 1.0 / sqrt(s) : 0.0;
    ai = 0;
  } else {
    ar = alpha[0];
    ai = alpha[1];
  }
  const T r = T(ar), i_ = T(ai);
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.x * NT) {
    cx<T> v = x[e];
    y[e] = mk<T>(r * v.re - i_ * v.im, r * v.im + i_ * v.re);
  }
}

template <typename TX, typename TY>
__global__ void __launch_bounds__(NT) k_convert(const cx<TX>* __restrict__ x, cx<TY>* __restrict__ y, size_t n) {
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.x * NT) y[e] = cvt<TY>(x[e]);
}

template <typename TX, typename TZ, typename TY>
__global__ void __launch_bounds__(NT) k_add(const cx<TX>* __restrict__ x, const cx<TZ>* __restrict__ z,
                                            cx<TY>* __restrict__ y, size_t n) {
  using T = typename std::conditional<(sizeof(TX) > sizeof(TZ)), TX, TZ>::type;
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.x * NT)
    y[e] = cvt<TY>(cvt<T>(x[e]) + cvt<T>(z[e]));
}

// y = A x with A dense complex double (row-major n x n); one warp per row; batch in blockIdx.y,
// right-hand side b with the matrix A + b astride (astride 0: one matrix for the batch)
template <typename T>
__global__ void __launch_bounds__(NT) k_dense(const cx<double>* __restrict__ A, size_t astride, int n,
                                              const cx<T>* __restrict__ x, cx<T>* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  const size_t off = (size_t)blockIdx.y * n;
  if (row >= n) return;
  A += blockIdx.y * astride;
  double sr = 0, si = 0;
  for (int c = lane; c < n; c += 32) {
    cx<double> a = A[(size_t)row * n + c];
    cx<double> v = cvt<double>(x[off + c]);
    sr += a.re * v.re - a.im * v.im;
    si += a.re * v.im + a.im * v.re;
  }
  sr = warp_sum(sr);
  si = warp_sum(si);
  if (lane == 0) y[off + row] = cvt<T>(mk<double>(sr, si));
}

inline unsigned g1(size_t n) {
  size_t b = (n + NT - 1) / NT;
  size_t cap = 152 * 8;
  return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

namespace hz {

size_t dot_ws_bytes(int nv, int nb) {
  return sizeof(double) * (size_t)MAXP * (2 * (size_t)(nv > 0 ? nv : 1) + 2) * (size_t)(nb > 0 ? nb : 1);
}

cudaError_t launch_multidot(Ctx& c, int dt, const void* V, size_t ldv, int nv, const void* w, size_t n, int nb,
                            double* out, void* ws, int with_norm, const double* skip) {
  if (nv <= 0) return cudaSuccess;
  int np = nparts(n);
  int ldp = 2 * nv + (with_norm ? 1 : 0);
  double* part = reinterpret_cast<double*>(ws);
  dim3 grid((nv + CV - 1) / CV, np, nb);
  {
    ProfScope ps(c, F_DOT, (double)nb * n * elem_bytes(dt) * (nv + 1));
    if (dt == C128)
      k_multidot<double><<<grid, NT, 0, c.s>>>(reinterpret_cast<const cx<double>*>(V), ldv, nv,
                                               reinterpret_cast<const cx<double>*>(w), n, part, ldp, with_norm, skip);
    else
      k_multidot<float><<<grid, NT, 0, c.s>>>(reinterpret_cast<const cx<float>*>(V), ldv, nv,
                                              reinterpret_cast<const cx<float>*>(w), n, part, ldp, with_norm, skip);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ProfScope ps2(c, F_REDUCE, (double)nb * np * ldp * 8);
  k_reduce<<<dim3(ldp, nb), NT, 0, c.s>>>(part, np, ldp, ldp, out);
  return cudaGetLastError();
}

cudaError_t launch_update(Ctx& c, int dtv, const void* V, size_t ldv, int nv, const double* coef, int ldc, int dtw,
                          void* w, size_t n, int nb, double* nrm2, void* ws, const double* skip) {
  unsigned np = (unsigned)nparts(n);
  double* part = nrm2 ? reinterpret_cast<double*>(ws) : nullptr;
  size_t sm = sizeof(double) * 2 * (size_t)(nv > 0 ? nv : 1);
  dim3 grid(np, nb);
  {
    ProfScope ps(c, F_AXPY, (double)nb * n * (elem_bytes(dtv) * nv + 2 * elem_bytes(dtw)));
    if (dtv == C128 && dtw == C128)
      k_update<double, double><<<grid, NT, sm, c.s>>>(reinterpret_cast<const cx<double>*>(V), ldv, nv, coef, ldc,
                                                      reinterpret_cast<cx<double>*>(w), n, part, skip);
    else if (dtv == C64 && dtw == C64)
      k_update<float, float><<<grid, NT, sm, c.s>>>(reinterpret_cast<const cx<float>*>(V), ldv, nv, coef, ldc,
                                                    reinterpret_cast<cx<float>*>(w), n, part, skip);
    else if (dtv == C128 && dtw == C64)
      k_update<double, float><<<grid, NT, sm, c.s>>>(reinterpret_cast<const cx<double>*>(V), ldv, nv, coef, ldc,
                                                     reinterpret_cast<cx<float>*>(w), n, part, skip);
    else
      k_update<float, double><<<grid, NT, sm, c.s>>>(reinterpret_cast<const cx<float>*>(V), ldv, nv, coef, ldc,
                                                     reinterpret_cast<cx<double>*>(w), n, part, skip);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !nrm2) return e;
  ProfScope ps2(c, F_REDUCE, (double)nb * np * 8);
  k_reduce<<<dim3(1, nb), NT, 0, c.s>>>(part, (int)np, 1, 1, nrm2);
  return cudaGetLastError();
}

cudaError_t launch_dgks_flag(Ctx& c, const double* wn, int ldw, const double* n1, double* flag, int nb, double eta2) {
  ProfScope ps(c, F_REDUCE, (double)nb * 24);
  k_dgks<<<(nb + 127) / 128, 128, 0, c.s>>>(wn, ldw, n1, flag, nb, eta2);
  return cudaGetLastError();
}

cudaError_t launch_row_scale(Ctx& c, int nx, int ny, const void* x, void* y, int nb) {
  const size_t n = (size_t)nx * ny;
  ProfScope ps(c, F_MISC, (double)nb * n * 32.0);
  const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
  k_row_scale<<<dim3(blocks, nb), 256, 0, c.s>>>(reinterpret_cast<const cx<double>*>(x), reinterpret_cast<cx<double>*>(y),
                                                 nx, ny);
  return cudaGetLastError();
}

cudaError_t launch_m1_mr(Ctx& c, const double* d, int nb, double* coef, int* its, int* calls, int* err) {
  ProfScope ps(c, F_REDUCE, 0.0);
  k_m1_mr<<<(nb + 127) / 128, 128, 0, c.s>>>(d, nb, coef, its, calls, err);
  return cudaGetLastError();
}

cudaError_t launch_combine(Ctx& c, int dtx, const void* X, size_t ldx, int nv, const double* coef, int dtu, void* u,
                           size_t n, int nb) {
  if (nv <= 0) return cudaSuccess;
  size_t sm = sizeof(double) * 2 * (size_t)nv;
  ProfScope ps(c, F_AXPY, (double)nb * n * (elem_bytes(dtx) * nv + 2 * elem_bytes(dtu)));
  dim3 grid(g1(n), nb);
  if (dtx == C128 && dtu == C128)
    k_combine<double, double><<<grid, NT, sm, c.s>>>(reinterpret_cast<const cx<double>*>(X), ldx, nv, coef,
                                                     reinterpret_cast<cx<double>*>(u), n);
  else if (dtx == C64 && dtu == C64)
    k_combine<float, float><<<grid, NT, sm, c.s>>>(reinterpret_cast<const cx<float>*>(X), ldx, nv, coef,
                                                   reinterpret_cast<cx<float>*>(u), n);
  else if (dtx == C64 && dtu == C128)
    k_combine<float, double><<<grid, NT, sm, c.s>>>(reinterpret_cast<const cx<float>*>(X), ldx, nv, coef,
                                                    reinterpret_cast<cx<double>*>(u), n);
  else
    k_combine<double, float><<<grid, NT, sm, c.s>>>(reinterpret_cast<const cx<double>*>(X), ldx, nv, coef,
                                                    reinterpret_cast<cx<float>*>(u), n);
  return cudaGetLastError();
}

cudaError_t launch_scale_dev(Ctx& c, int dt, const void* x, void* y, const double* alpha_dev, int recip, size_t n,
                             int nb) {
  ProfScope ps(c, F_AXPY, (double)nb * n * 2 * elem_bytes(dt));
  dim3 grid(g1(n), nb);
  if (dt == C128)
    k_scale<double><<<grid, NT, 0, c.s>>>(reinterpret_cast<const cx<double>*>(x), reinterpret_cast<cx<double>*>(y),
                                          alpha_dev, recip, n);
  else
    k_scale<float><<<grid, NT, 0, c.s>>>(reinterpret_cast<const cx<float>*>(x), reinterpret_cast<cx<float>*>(y),
                                         alpha_dev, recip, n);
  return cudaGetLastError();
}

cudaError_t launch_convert(Ctx& c, int tx, int ty, const void* x, void* y, size_t n) {
  ProfScope ps(c, F_MISC, (double)n * (elem_bytes(tx) + elem_bytes(ty)));
  if (tx == C128 && ty == C64)
    k_convert<double, float><<<g1(n), NT, 0, c.s>>>(reinterpret_cast<const cx<double>*>(x), reinterpret_cast<cx<float>*>(y), n);
  else if (tx == C64 && ty == C128)
    k_convert<float, double><<<g1(n), NT, 0, c.s>>>(reinterpret_cast<const cx<float>*>(x), reinterpret_cast<cx<double>*>(y), n);
  else
    return cudaMemcpyAsync(y, x, n * elem_bytes(tx), cudaMemcpyDeviceToDevice, c.s);
  return cudaGetLastError();
}

cudaError_t launch_add(Ctx& c, int tx, const void* x, int tz, const void* z, int ty, void* y, size_t n) {
  ProfScope ps(c, F_MISC, (double)n * (elem_bytes(tx) + elem_bytes(tz) + elem_bytes(ty)));
#define HZ_ADD(A, B, C)                                                                                      \
  k_add<A, B, C><<<g1(n), NT, 0, c.s>>>(reinterpret_cast<const cx<A>*>(x), reinterpret_cast<const cx<B>*>(z), \
                                        reinterpret_cast<cx<C>*>(y), n)
  if (tx == C64 && tz == C64 && ty == C64) HZ_ADD(float, float, float);
  else if (tx == C128 && tz == C128 && ty == C128) HZ_ADD(double, double, double);
  else if (tx == C64 && tz == C64 && ty == C128) HZ_ADD(float, float, double);
  else return cudaErrorInvalidValue;
#undef HZ_ADD
  return cudaGetLastError();
}

cudaError_t launch_dense(Ctx& c, const double* A, int n, int dt, const void* x, void* y, int nrhs, size_t astride) {
  dim3 grid((n + NT / 32 - 1) / (NT / 32), nrhs);
  ProfScope ps(c, F_DENSE, (double)n * n * 16.0 * (astride ? nrhs : 1));
  if (dt == C128)
    k_dense<double><<<grid, NT, 0, c.s>>>(reinterpret_cast<const cx<double>*>(A), astride, n,
                                          reinterpret_cast<const cx<double>*>(x), reinterpret_cast<cx<double>*>(y));
  else
    k_dense<float><<<grid, NT, 0, c.s>>>(reinterpret_cast<const cx<double>*>(A), astride, n,
                                         reinterpret_cast<const cx<float>*>(x), reinterpret_cast<cx<float>*>(y));
  return cudaGetLastError();
}

}  // namespace hz
