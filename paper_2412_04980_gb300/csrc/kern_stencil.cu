// Stencil kernels of the hot path: level operators (Section 2.1, Section 3.3), deflation
// transfers Z / Z^T (Section 3.1, Algorithm 1 lines 5 and 11-13) and the multigrid
// CSLP pieces (damped Jacobi, full weighting, bilinear prolongation).
//
// Every kernel is HBM-bound in FP32 and FP64-ALU-bound in FP64 on this part; inputs are
// staged once per CTA in shared memory (tile + halo), outputs are written coalesced.
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>

#include "hz_device.cuh"
#include "hz_internal.h"

using namespace hzd;

namespace {

constexpr int BX = 32, BY = 8;          // 256 threads per CTA
constexpr int OXT = 32, OYT = 16;       // output tile of the fine-grid kernels

__host__ __device__ inline int floordiv2(int a) { return (a >= 0) ? (a >> 1) : -((-a + 1) >> 1); }

// Coarse nodes per side: vertex grids keep both boundary nodes, (n + 1) / 2; Dirichlet grids hold
// interior unknowns only, (n - 1) / 2.
inline int coarse_n(int n, int bc) { return bc != 0 ? (n - 1) / 2 : (n + 1) / 2; }

template <typename T>
OpP<T> make_op(const hz::OpDesc& d) {
  OpP<T> p;
  p.nx = d.nx;
  p.ny = d.ny;
  p.R = d.R;
  p.bc = d.bc;
  p.srow = d.srow;
  p.c = T(d.c);
  p.H = T(d.H);
  p.ks = T(d.ks);
  p.sr = T(d.sr);
  p.si = T(d.si);
  p.ksr = T(d.ks * d.sr);
  p.ksi = T(d.ks * d.si);
  for (int i = 0; i < 7; ++i) {
    p.m[i] = T(d.m[i]);
    p.l[i] = T(d.l[i]);
  }
  if constexpr (sizeof(T) == 8) p.k = reinterpret_cast<const T*>(d.k_d);
  else p.k = reinterpret_cast<const T*>(d.k_f);
  p.kstride = d.kstride;
  return p;
}

template <typename T>
__device__ __forceinline__ T pw(int d) {  // deflation weights p = [1,4,6,4,1]/8
  return d == 0 ? T(0.75) : ((d == 1 || d == -1) ? T(0.5) : ((d == 2 || d == -2) ? T(0.125) : T(0)));
}

template <typename T, typename TI>
struct GlobalSrc {
  const cx<TI>* x;
  int nx;
  __device__ __forceinline__ cx<T> operator()(int gx, int gy) const { return cvt<T>(x[(size_t)gy * nx + gx]); }
};

// omega * f / D : one Jacobi sweep from a zero initial guess
template <typename T, int R>
struct JacZeroSrc {
  const cx<T>* f;
  OpP<T> P;
  T omega;
  __device__ __forceinline__ cx<T> operator()(int gx, int gy) const {
    return omega * cdiv(f[(size_t)gy * P.nx + gx], op_diag<T, R>(P, gx, gy));
  }
};

// omega f / D + bilinear(ec) from a coarse tile in shared memory
template <typename T, int R>
struct UpSrc {
  const cx<T>* f;
  OpP<T> P;
  T omega;
  const cx<T>* Es;
  int EW, Imin, Jmin, dof;  // dof = 1 on Dirichlet grids (coarse unknown I at fine unknown 2I + 1)
  __device__ __forceinline__ cx<T> operator()(int gx, int gy) const {
    cx<T> u = omega * cdiv(f[(size_t)gy * P.nx + gx], op_diag<T, R>(P, gx, gy));
    int I = floordiv2(gx + dof), J = floordiv2(gy + dof);
    int ex = gx + dof - 2 * I, ey = gy + dof - 2 * J;
    const cx<T>* e = Es + (J - Jmin) * EW + (I - Imin);
    cx<T> a = e[0];
    if (ex) a = T(0.5) * (a + e[1]);
    if (ey) {
      cx<T> b = e[EW];
      if (ex) b = T(0.5) * (b + e[EW + 1]);
      a = T(0.5) * (a + b);
    }
    return u + a;
  }
};

// The radius-1 row of tile_op at tile cell (ox, oy) with the node's wavenumber k given (loaded by
// the caller ahead of the tile barrier); same arithmetic as tile_op.
template <typename T>
__device__ __forceinline__ cx<T> op1_k(const TileView<T, 1>& t, const OpP<T>& P, int ox, int oy, T k) {
  const int WX = t.WX();
  const cx<T>* uc = t.U + (oy + 1) * WX + (ox + 1);
  const cx<T> s = (uc[1] + uc[-1]) + (uc[WX] + uc[-WX]);
  const T k2 = k * k;
  const T dr = fma(-P.ksr, k2, T(4) * P.c);
  const T di = P.ksi * k2;
  const cx<T> u = *uc;
  cx<T> v = mk<T>(fma(dr, u.re, fma(di, u.im, -P.c * s.re)), fma(dr, u.im, fma(-di, u.re, -P.c * s.im)));
  if (P.srow) {
    const int g = bsides(P, t.ox0 + ox, t.oy0 + oy);
    if (g) v = (g == 1 ? T(0.5) : T(0.25)) * v;
  }
  return v;
}

// ---------------------------------------------------------------------------------------
template <typename T, typename TI, typename TO, int R, int MODE>
__global__ void __launch_bounds__(BX* BY) k_level_op(OpP<T> P, const cx<TI>* __restrict__ x,
                                                       const cx<TI>* __restrict__ f, cx<TO>* __restrict__ y,
                                                       T omega) {
  P.k += (size_t)blockIdx.z * P.kstride;  // this right-hand side's wavenumber field
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t off = (size_t)blockIdx.z * P.nx * P.ny;
  x += off;
  y += off;
  if (MODE != 0) f += off;
  const int ox0 = blockIdx.x * OXT, oy0 = blockIdx.y * OYT;
  TileView<T, R> t = make_tile<T, R>(smem, OXT, OYT, ox0, oy0);
  // fi: f at the node (modes 1 and 2)
  auto emit = [&](int ox, int oy, cx<T> v, cx<T> fi) {
    const int gx = ox0 + ox, gy = oy0 + oy;
    const size_t i = (size_t)gy * P.nx + gx;
    cx<T> out;
    if (MODE == 0) {
      out = v;
    } else {
      cx<T> r = fi - v;
      if (MODE == 1) out = r;
      else out = t.u(ox + R, oy + R) + omega * cdiv(r, op_diag<T, R>(P, gx, gy));
    }
    y[i] = cvt<TO>(out);
  };
  if constexpr (R == 1) {
    // the wavenumbers (and f) of this thread's outputs are loaded with the staged values, ahead
    // of the tile barrier: one round of global-load latency per tile instead of two
    constexpr int NP = OYT / BY;
    T kr[NP];
    cx<T> fr[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int gx = ox0 + threadIdx.x, gy = oy0 + threadIdx.y + p * BY;
      const bool in = gx < P.nx && gy < P.ny;
      const size_t i = (size_t)gy * P.nx + gx;
      kr[p] = in ? __ldg(P.k + i) : T(0);
      fr[p] = (MODE != 0 && in) ? cvt<T>(f[i]) : mk<T>(T(0), T(0));
    }
    tile_fill<T, R>(t, P, GlobalSrc<T, TI>{x, P.nx});
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int ox = threadIdx.x, oy = threadIdx.y + p * BY;
      if (ox0 + ox >= P.nx || oy0 + oy >= P.ny) continue;
      emit(ox, oy, op1_k<T>(t, P, ox, oy, kr[p]), fr[p]);
    }
  } else {
    tile_fill<T, R>(t, P, GlobalSrc<T, TI>{x, P.nx});
    const int tid = threadIdx.y * BX + threadIdx.x;
    constexpr int SEG = R == 2 ? 2 : 4;
    for (int it = tid; it < OXT * (OYT / SEG); it += BX * BY) {
      const int ox = it % OXT, sy = (it / OXT) * SEG;
      const int cnt = min(SEG, P.ny - (oy0 + sy));
      if (ox0 + ox >= P.nx || cnt <= 0) continue;
      cx<T> v[4];
      tile_op_seg<T, R, SEG>(t, P, ox, sy, cnt, v);
      for (int q = 0; q < cnt; ++q) {
        const size_t i = (size_t)(oy0 + sy + q) * P.nx + ox0 + ox;
        emit(ox, sy + q, v[q], MODE != 0 ? cvt<T>(f[i]) : mk<T>(T(0), T(0)));
      }
    }
  }
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_jacobi_zero(OpP<T> P, const cx<T>* __restrict__ f, cx<T>* __restrict__ y,
                                                     T omega) {
  P.k += (size_t)blockIdx.y * P.kstride;  // this right-hand side's wavenumber field
  const size_t n = (size_t)P.nx * P.ny;
  const size_t off = (size_t)blockIdx.y * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int gy = (int)(i / P.nx), gx = (int)(i - (size_t)gy * P.nx);
    y[off + i] = omega * cdiv(f[off + i], op_diag<T, R>(P, gx, gy));
  }
}

// t = Z vtil ; rtil = v - A t  (Algorithm 1, lines 11-13)
template <typename T, typename TV, int R>
__global__ void __launch_bounds__(BX* BY) k_defl_prolong_resid(OpP<T> P, const cx<T>* __restrict__ vtil, int ncx,
                                                                 int ncy, const cx<TV>* __restrict__ v,
                                                                 cx<T>* __restrict__ tout, cx<T>* __restrict__ rtil) {
  P.k += (size_t)blockIdx.z * P.kstride;  // this right-hand side's wavenumber field
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t off = (size_t)blockIdx.z * P.nx * P.ny;
  const size_t offc = (size_t)blockIdx.z * ncx * ncy;
  const int ox0 = blockIdx.x * OXT, oy0 = blockIdx.y * OYT;
  // coarse indices below are those of the vertex grid; on a Dirichlet grid (dof = 1) fine unknown
  // g is vertex g + 1 and coarse unknown I is vertex I + 1 (its boundary vertices hold zero)
  const int dof = P.bc != 0;
  const int Imin = floordiv2(ox0 + dof - R - 1), Imax = floordiv2(ox0 + dof + OXT + R + 1);
  const int Jmin = floordiv2(oy0 + dof - R - 1), Jmax = floordiv2(oy0 + dof + OYT + R + 1);
  const int CW = Imax - Imin + 1, CH = Jmax - Jmin + 1;
  TileView<T, R> t = make_tile<T, R>(smem, OXT, OYT, ox0, oy0);
  cx<T>* Cs = reinterpret_cast<cx<T>*>(smem + tile_smem_bytes<T, R>(OXT, OYT));
  const int tid = threadIdx.y * BX + threadIdx.x;
  for (int idx = tid; idx < CW * CH; idx += BX * BY) {
    int cj = idx / CW, ci = idx - cj * CW;
    int I = Imin + ci - dof, J = Jmin + cj - dof;
    Cs[idx] = (I >= 0 && I < ncx && J >= 0 && J < ncy) ? vtil[offc + (size_t)J * ncx + I] : mk<T>(T(0), T(0));
  }
  __syncthreads();
  // t = Z vtil on the tile window, separably: the 1-D weights are 1/8, 3/4, 1/8 at even fine
  // nodes (coarse I-1, I, I+1) and 1/2, 1/2 at odd ones (I, I+1).  First every coarse row is
  // interpolated to the fine columns (Xs), then the columns to the fine rows (zero outside the grid).
  {
    constexpr int WX = OXT + 2 * R, WY = OYT + 2 * R;
    constexpr int CWM = (OXT + 2 * R + 6) / 2 + 2, CHM = (OYT + 2 * R + 6) / 2 + 2;
    cx<T>* Xs = Cs + CWM * CHM;
    const int gx0 = ox0 - R, gy0 = oy0 - R;
    for (int idx = tid; idx < CH * WX; idx += BX * BY) {
      const int cj = idx / WX, cxx = idx - cj * WX;
      const int gx = gx0 + cxx + dof;
      const cx<T>* r = Cs + cj * CW + (floordiv2(gx) - Imin);
      Xs[idx] = (gx & 1) ? T(0.5) * (r[0] + r[1]) : T(0.75) * r[0] + T(0.125) * (r[-1] + r[1]);
    }
    __syncthreads();
    for (int idx = tid; idx < WX * WY; idx += BX * BY) {
      const int cy = idx / WX, cxx = idx - cy * WX;
      const int gx = gx0 + cxx, gy = gy0 + cy;
      cx<T> u = mk<T>(T(0), T(0)), w = u;
      if (gx >= 0 && gx < P.nx && gy >= 0 && gy < P.ny) {
        const int ge = gy + dof;
        const cx<T>* c = Xs + (floordiv2(ge) - Jmin) * WX + cxx;
        u = (ge & 1) ? T(0.5) * (c[0] + c[WX]) : T(0.75) * c[0] + T(0.125) * (c[-WX] + c[WX]);
        if (R >= 2) {
          const T k = P.k[(size_t)gy * P.nx + gx];
          w = (k * k) * u;
        }
      }
      t.U[idx] = u;
      if (R >= 2) t.W[idx] = w;
    }
    __syncthreads();
    tile_finish<T, R>(t, P);
  }
  auto emit = [&](int ox, int oy, cx<T> s) {
    const size_t i = off + (size_t)(oy0 + oy) * P.nx + (ox0 + ox);
    rtil[i] = cvt<T>(v[i]) - s;
    if (tout) tout[i] = t.u(ox + R, oy + R);
  };
  if (R == 1) {
#pragma unroll
    for (int p = 0; p < OYT / BY; ++p) {
      const int ox = threadIdx.x, oy = threadIdx.y + p * BY;
      if (ox0 + ox >= P.nx || oy0 + oy >= P.ny) continue;
      emit(ox, oy, tile_op<T, R>(t, P, ox, oy));
    }
  } else {
    constexpr int SEG = R == 2 ? 2 : 4;
    for (int it = tid; it < OXT * (OYT / SEG); it += BX * BY) {
      const int ox = it % OXT, sy = (it / OXT) * SEG;
      const int cnt = min(SEG, P.ny - (oy0 + sy));
      if (ox0 + ox >= P.nx || cnt <= 0) continue;
      cx<T> sv[4];
      tile_op_seg<T, R, SEG>(t, P, ox, sy, cnt, sv);
      for (int q = 0; q < cnt; ++q) emit(ox, sy + q, sv[q]);
    }
  }
}

// plain t = Z w (Algorithm 1, line 11)
template <typename T>
__global__ void __launch_bounds__(256) k_defl_prolong(const cx<T>* __restrict__ w, int ncx, int ncy,
                                                      cx<T>* __restrict__ t, int nx, int ny, int dof) {
  const size_t n = (size_t)nx * ny;
  const size_t off = (size_t)blockIdx.y * n, offc = (size_t)blockIdx.y * ncx * ncy;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    // vertex-grid coordinates (dof = 1 on Dirichlet grids: unknown g is vertex g + 1)
    int gy = (int)(i / nx) + dof, gx = (int)(i % nx) + dof;
    int I0 = floordiv2(gx - 1), I1 = floordiv2(gx + 2), J0 = floordiv2(gy - 1), J1 = floordiv2(gy + 2);
    cx<T> acc = mk<T>(T(0), T(0));
    for (int J = J0; J <= J1; ++J) {
      if (J - dof < 0 || J - dof >= ncy) continue;
      cx<T> row = mk<T>(T(0), T(0));
      for (int I = I0; I <= I1; ++I) {
        if (I - dof < 0 || I - dof >= ncx) continue;
        row = row + pw<T>(gx - 2 * I) * w[offc + (size_t)(J - dof) * ncx + (I - dof)];
      }
      acc = acc + pw<T>(gy - 2 * J) * row;
    }
    t[off + i] = acc;
  }
}

// vhat = Z^T v (Algorithm 1, line 5): separable 5-tap filters at stride 2
constexpr int RXC = 32, RYC = 16;
template <typename TI, typename T>
__global__ void __launch_bounds__(BX* BY) k_defl_restrict(const cx<TI>* __restrict__ v, int nx, int ny,
                                                            cx<T>* __restrict__ vhat, int ncx, int ncy, int dof) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int FW = 2 * RXC + 3, FH = 2 * RYC + 3;
  cx<T>* F = reinterpret_cast<cx<T>*>(smem);
  cx<T>* XR = F + FW * FH;
  const size_t off = (size_t)blockIdx.z * nx * ny, offc = (size_t)blockIdx.z * ncx * ncy;
  const int x0c = blockIdx.x * RXC, y0c = blockIdx.y * RYC;
  // coarse unknown I is centred on fine unknown 2I + dof (dof = 1 on Dirichlet grids)
  const int fx0 = 2 * x0c - 2 + dof, fy0 = 2 * y0c - 2 + dof;
  const int tid = threadIdx.y * BX + threadIdx.x;
  for (int idx = tid; idx < FW * FH; idx += BX * BY) {
    int fy = idx / FW, fx = idx - fy * FW;
    int gx = fx0 + fx, gy = fy0 + fy;
    F[idx] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? cvt<T>(v[off + (size_t)gy * nx + gx]) : mk<T>(T(0), T(0));
  }
  __syncthreads();
  for (int idx = tid; idx < FH * RXC; idx += BX * BY) {
    int fy = idx / RXC, ox = idx - fy * RXC;
    const cx<T>* r = F + fy * FW + 2 * ox;   // fine cell 2*ox + 2 + a at r[2 + a]
    XR[idx] = (T(0.125) * (r[0] + r[4]) + T(0.5) * (r[1] + r[3])) + T(0.75) * r[2];
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < RYC / BY; ++p) {
    int ox = threadIdx.x, oy = threadIdx.y + p * BY;
    int I = x0c + ox, J = y0c + oy;
    if (I >= ncx || J >= ncy) continue;
    const cx<T>* c = XR + (2 * oy) * RXC + ox;   // fine row 2*oy + 2 + b at c[(2 + b) * RXC]
    vhat[offc + (size_t)J * ncx + I] =
        (T(0.125) * (c[0] + c[4 * RXC]) + T(0.5) * (c[RXC] + c[3 * RXC])) + T(0.75) * c[2 * RXC];
  }
}

// fc = FW(f - Op(omega f / D)) : pre-smoothing from zero, residual, full weighting
constexpr int DXC = 32, DYC = 8;
template <typename T, int R>
__global__ void __launch_bounds__(BX* BY) k_mg_down(OpP<T> P, const cx<T>* __restrict__ f, cx<T>* __restrict__ fc,
                                                      int ncx, int ncy, T omega) {
  P.k += (size_t)blockIdx.z * P.kstride;  // this right-hand side's wavenumber field
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int OX = 2 * DXC + 1, OY = 2 * DYC + 1;
  const size_t off = (size_t)blockIdx.z * P.nx * P.ny, offc = (size_t)blockIdx.z * ncx * ncy;
  f += off;
  const int x0c = blockIdx.x * DXC, y0c = blockIdx.y * DYC;
  // full weighting centred on fine node 2I (2I + 1 on Dirichlet grids)
  const int dof = P.bc != 0;
  const int ox0 = 2 * x0c - 1 + dof, oy0 = 2 * y0c - 1 + dof;
  TileView<T, R> t = make_tile<T, R>(smem, OX, OY, ox0, oy0);
  cx<T>* RS = reinterpret_cast<cx<T>*>(smem + tile_smem_bytes<T, R>(OX, OY));
  tile_fill<T, R>(t, P, JacZeroSrc<T, R>{f, P, omega});
  const int tid = threadIdx.y * BX + threadIdx.x;
  if (R == 1) {
    for (int idx = tid; idx < OX * OY; idx += BX * BY) {
      int oy = idx / OX, ox = idx - oy * OX;
      int gx = ox0 + ox, gy = oy0 + oy;
      cx<T> r = mk<T>(T(0), T(0));
      if (gx >= 0 && gx < P.nx && gy >= 0 && gy < P.ny) r = f[(size_t)gy * P.nx + gx] - tile_op<T, R>(t, P, ox, oy);
      RS[idx] = r;
    }
  } else {
    constexpr int SEG = R == 2 ? 2 : 4;
    constexpr int NSY = (OY + SEG - 1) / SEG;
    for (int it = tid; it < OX * NSY; it += BX * BY) {
      const int ox = it % OX, sy = (it / OX) * SEG;
      const int cnt = min(SEG, OY - sy);
      const int gx = ox0 + ox;
      // rows of this segment that lie in the grid
      int q0 = 0, q1 = cnt;
      while (q0 < cnt && oy0 + sy + q0 < 0) ++q0;
      while (q1 > q0 && oy0 + sy + q1 - 1 >= P.ny) --q1;
      cx<T> v[4];
      const bool colok = gx >= 0 && gx < P.nx;
      if (colok && q1 > q0) {
        cx<T> w4[4];
        tile_op_seg<T, R, SEG>(t, P, ox, sy + q0, q1 - q0, w4);
        for (int q = q0; q < q1; ++q) v[q] = w4[q - q0];
      }
      for (int q = 0; q < cnt; ++q) {
        const int gy = oy0 + sy + q;
        cx<T> r = mk<T>(T(0), T(0));
        if (colok && q >= q0 && q < q1) r = f[(size_t)gy * P.nx + gx] - v[q];
        RS[(sy + q) * OX + ox] = r;
      }
    }
  }
  __syncthreads();
  const int ox = threadIdx.x, oy = threadIdx.y;
  const int I = x0c + ox, J = y0c + oy;
  if (I < ncx && J < ncy) {
    const cx<T>* c = RS + (2 * oy + 1) * OX + (2 * ox + 1);
    cx<T> s = (T(4) * c[0] + T(2) * ((c[1] + c[-1]) + (c[OX] + c[-OX]))) +
              ((c[OX + 1] + c[OX - 1]) + (c[-OX + 1] + c[-OX - 1]));
    fc[offc + (size_t)J * ncx + I] = T(0.0625) * s;
  }
}

// u = omega f / D + P ec ; y = u + omega (f - Op u) / D [+ add]
template <typename T, int R>
__global__ void __launch_bounds__(BX* BY) k_mg_up(OpP<T> P, const cx<T>* __restrict__ f, const cx<T>* __restrict__ ec,
                                                    int ncx, int ncy, cx<T>* __restrict__ y, T omega,
                                                    const cx<T>* __restrict__ add) {
  P.k += (size_t)blockIdx.z * P.kstride;  // this right-hand side's wavenumber field
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t off = (size_t)blockIdx.z * P.nx * P.ny, offc = (size_t)blockIdx.z * ncx * ncy;
  f += off;
  const int ox0 = blockIdx.x * OXT, oy0 = blockIdx.y * OYT;
  // vertex-grid coarse indices (Dirichlet: fine unknown g is vertex g + 1, coarse I is vertex I + 1)
  const int dof = P.bc != 0;
  const int Imin = floordiv2(ox0 + dof - R), Imax = floordiv2(ox0 + dof + OXT + R - 1) + 1;
  const int Jmin = floordiv2(oy0 + dof - R), Jmax = floordiv2(oy0 + dof + OYT + R - 1) + 1;
  const int EW = Imax - Imin + 1, EH = Jmax - Jmin + 1;
  TileView<T, R> t = make_tile<T, R>(smem, OXT, OYT, ox0, oy0);
  cx<T>* Es = reinterpret_cast<cx<T>*>(smem + tile_smem_bytes<T, R>(OXT, OYT));
  const int tid = threadIdx.y * BX + threadIdx.x;
  for (int idx = tid; idx < EW * EH; idx += BX * BY) {
    int cj = idx / EW, ci = idx - cj * EW;
    int I = Imin + ci - dof, J = Jmin + cj - dof;
    Es[idx] = (I >= 0 && I < ncx && J >= 0 && J < ncy) ? ec[offc + (size_t)J * ncx + I] : mk<T>(T(0), T(0));
  }
  __syncthreads();
  tile_fill<T, R>(t, P, UpSrc<T, R>{f, P, omega, Es, EW, Imin, Jmin, dof});
  auto emit = [&](int ox, int oy, cx<T> val) {
    const int gx = ox0 + ox, gy = oy0 + oy;
    const size_t i = (size_t)gy * P.nx + gx;
    cx<T> r = f[i] - val;
    cx<T> out = t.u(ox + R, oy + R) + omega * cdiv(r, op_diag<T, R>(P, gx, gy));
    if (add) out = out + add[off + i];
    y[off + i] = out;
  };
  if (R == 1) {
#pragma unroll
    for (int p = 0; p < OYT / BY; ++p) {
      const int ox = threadIdx.x, oy = threadIdx.y + p * BY;
      if (ox0 + ox >= P.nx || oy0 + oy >= P.ny) continue;
      emit(ox, oy, tile_op<T, R>(t, P, ox, oy));
    }
  } else {
    constexpr int SEG = R == 2 ? 2 : 4;
    for (int it = tid; it < OXT * (OYT / SEG); it += BX * BY) {
      const int ox = it % OXT, sy = (it / OXT) * SEG;
      const int cnt = min(SEG, P.ny - (oy0 + sy));
      if (ox0 + ox >= P.nx || cnt <= 0) continue;
      cx<T> v[4];
      tile_op_seg<T, R, SEG>(t, P, ox, sy, cnt, v);
      for (int q = 0; q < cnt; ++q) emit(ox, sy + q, v[q]);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Radius-1 multigrid sweeps as column strips.  A warp owns 64 consecutive grid columns, two per
// lane, and walks down a band of rows keeping a window of rows in registers; a lane's own pair
// supplies one horizontal neighbour of each of its nodes and the adjacent lanes the other (one
// shuffle each way), so the sweep needs no shared-memory tile and no per-node index arithmetic.
// The first and last lane of a warp only supply neighbours (the strips of adjacent warps overlap
// by two columns on each side and compute those twice).
//
// With the radius-1 operator M u = D u - c S(u), D the exact diagonal (ghost feedback included)
// and S(u) the sum of the four neighbours with the Sommerfeld ghost replaced by the inner
// neighbour (its boundary term is in D), the pre-smoothed residual of the zero initial guess
// u0 = omega f / D is r = f - M u0 = (1 - omega) f + c S(u0), and the post-smoothing step
// y = u + omega (f - M u) / D with u = u0 + e is y = (1 - omega) u + u0 + omega c S(u) / D.
template <typename T>
__device__ __forceinline__ T r1_recip(T x) {
  if constexpr (sizeof(T) == 4) return __fdividef(1.f, x);  // FP32 sweeps: approximate reciprocal
  else return T(1) / x;
}

// Per-lane column data of one of the lane's two columns.
struct R1Col {
  int g;       // grid column
  bool in;     // inside the grid
  int bnd;     // 1 on the left or right boundary column (Sommerfeld)
};

template <typename T>
struct R1Ops {  // operator constants in the sweep's type
  T c4, ksr, ksi, c2H, c;
  int bc, nx, ny;
  __device__ __forceinline__ void diag(T kk, int g, T& dr, T& di) const {  // D at a node on g boundary sides
    const T k2 = kk * kk;
    dr = fma(-ksr, k2, c4);
    di = -ksi * k2;
    if (g) di -= c2H * kk * T(g);
  }
};

// fc = FW(f - M(omega f / D)) on the coarse grid; coarse node I sits at fine node 2I + dof.
// Strip s, lane L: coarse column I = 30 s + L - 1 at fine columns 2I + dof (a) and 2I + dof + 1
// (b); outputs at lanes 1 .. 30.  Band: coarse rows J0 .. J0 + RB - 1.  A warp whose window
// touches no boundary row or column (IN) runs without in-grid tests and ghost handling.
constexpr int kPF = 3;  // rows of loads in flight per lane
template <typename T, bool IN>
__device__ __forceinline__ void mg_down_band(const OpP<T>& P, const cx<T>* __restrict__ f, cx<T>* __restrict__ fcz,
                                             int ncx, int ncy, T omega, int I, int J0, int RB, int lane) {
  const int dof = P.bc != 0;
  const bool som = !IN && P.bc == 0;
  const T c4 = T(4) * P.c, c2H = P.c * T(2) * P.H, om1 = T(1) - omega;
  const int ga = 2 * I + dof, gb = ga + 1;
  const bool ain = IN || (ga >= 0 && ga < P.nx), bin = IN || (gb >= 0 && gb < P.nx);
  const int abnd = som && ain && (ga == 0 || ga == P.nx - 1), bbnd = som && bin && (gb == 0 || gb == P.nx - 1);
  const int yb = 2 * J0 + dof - 2, ye = 2 * (J0 + RB) + dof;
  // lane pointers to columns a and b of row yb (clamped for lanes outside the grid)
  const cx<T>* fp = f + (size_t)max(yb, 0) * P.nx + max(min(ga, P.nx - 2), 0);
  const T* kp = P.k + (size_t)max(yb, 0) * P.nx + max(min(ga, P.nx - 2), 0);
  const int fda = ga - max(min(ga, P.nx - 2), 0);  // 0, or -1 / +1 ... for clamped edge lanes
  auto load = [&](int gy, cx<T>& fa, cx<T>& fb, T& ka, T& kb) {
    if (IN) {
      const size_t o = (size_t)(gy - yb) * P.nx;
      fa = fp[o];
      fb = fp[o + 1];
      ka = kp[o];
      kb = kp[o + 1];
    } else {
      const bool rin = gy >= 0 && gy < P.ny;
      const size_t o = (size_t)(gy - max(yb, 0)) * P.nx;
      fa = (rin && ain) ? fp[o + fda] : mk<T>(T(0), T(0));
      fb = (rin && bin) ? fp[o + fda + 1] : mk<T>(T(0), T(0));
      ka = (rin && ain) ? kp[o + fda] : T(0);
      kb = (rin && bin) ? kp[o + fda + 1] : T(0);
    }
  };
  auto smooth0 = [&](bool cin, int cbnd, int gy, cx<T> fv, T kv) -> cx<T> {  // u0 = omega f / D
    if (!IN && !(cin && gy >= 0 && gy < P.ny)) return mk<T>(T(0), T(0));
    const T k2 = kv * kv;
    const T dr = fma(-P.ksr, k2, c4);
    T di = -P.ksi * k2;
    if (som) {
      const int g = cbnd + (gy == 0 || gy == P.ny - 1);
      if (g) di -= c2H * kv * T(g);
    }
    const T inv = omega * r1_recip<T>(dr * dr + di * di);
    return mk<T>((fv.re * dr + fv.im * di) * inv, (fv.im * dr - fv.re * di) * inv);
  };
  cx<T> fa_m1 = mk<T>(T(0), T(0)), fb_m1 = fa_m1;
  cx<T> ua_m2 = fa_m1, ub_m2 = fa_m1, ua_m1 = fa_m1, ub_m1 = fa_m1;
  cx<T> rhA = fa_m1, rhB = fa_m1;
  cx<T> pfa[kPF], pfb[kPF];
  T pka[kPF], pkb[kPF];
#pragma unroll
  for (int q = 0; q < kPF; ++q) load(yb + q, pfa[q], pfb[q], pka[q], pkb[q]);
  for (int y0 = yb; y0 <= ye; y0 += kPF) {
#pragma unroll
    for (int q = 0; q < kPF; ++q) {
      const int y = y0 + q;
      if (y > ye) break;
      const cx<T> fa = pfa[q], fb = pfb[q];
      const T ka = pka[q], kb = pkb[q];
      if (y + kPF <= ye) load(y + kPF, pfa[q], pfb[q], pka[q], pkb[q]);
      const cx<T> ua = smooth0(ain, abnd, y, fa, ka), ub = smooth0(bin, bbnd, y, fb, kb);
      if (y >= yb + 2) {
        const int yr = y - 1;  // residual row: u0 rows yr - 1 (m2), yr (m1), yr + 1 (this)
        cx<T> wa = mk<T>(__shfl_up_sync(0xffffffffu, ub_m1.re, 1), __shfl_up_sync(0xffffffffu, ub_m1.im, 1));
        cx<T> eb = mk<T>(__shfl_down_sync(0xffffffffu, ua_m1.re, 1), __shfl_down_sync(0xffffffffu, ua_m1.im, 1));
        cx<T> ea = ub_m1, wb = ua_m1;
        cx<T> sa = ua_m2, na = ua, sb = ub_m2, nb = ub;
        if (som) {  // ghosts take the inner neighbour
          if (ga == 0) wa = ea;
          if (ga == P.nx - 1) ea = wa;
          if (gb == 0) wb = eb;
          if (gb == P.nx - 1) eb = wb;
          if (yr == 0) {
            sa = na;
            sb = nb;
          }
          if (yr == P.ny - 1) {
            na = sa;
            nb = sb;
          }
        }
        cx<T> ra = om1 * fa_m1 + P.c * ((wa + ea) + (sa + na));
        cx<T> rb = om1 * fb_m1 + P.c * ((wb + eb) + (sb + nb));
        if (!IN) {
          const bool rin = yr >= 0 && yr < P.ny;
          if (!(rin && ain)) ra = mk<T>(T(0), T(0));
          if (!(rin && bin)) rb = mk<T>(T(0), T(0));
        }
        // horizontal full weighting 1 2 1 centred on column a: r(a - 1) is the previous lane's rb
        const cx<T> rw = mk<T>(__shfl_up_sync(0xffffffffu, rb.re, 1), __shfl_up_sync(0xffffffffu, rb.im, 1));
        const cx<T> rh = (rw + rb) + T(2) * ra;
        if (((yr - dof) & 1) != 0) {  // row 2J + dof + 1 (or the band's first row 2 J0 + dof - 1)
          if (yr > 2 * J0 + dof - 1) {
            const int J = (yr - dof - 1) / 2;
            if (lane >= 1 && lane <= 30 && I < ncx && J < ncy) fcz[(size_t)J * ncx + I] = T(0.0625) * ((rhA + rh) + T(2) * rhB);
          }
          rhA = rh;
        } else {
          rhB = rh;
        }
      }
      fa_m1 = fa;
      fb_m1 = fb;
      ua_m2 = ua_m1;
      ub_m2 = ub_m1;
      ua_m1 = ua;
      ub_m1 = ub;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_mg_down_r1(OpP<T> P, const cx<T>* __restrict__ f, cx<T>* __restrict__ fc,
                                                    int ncx, int ncy, T omega, int RB) {
  P.k += (size_t)blockIdx.z * P.kstride;  // this right-hand side's wavenumber field
  const int lane = threadIdx.x & 31;
  const int strip = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (30 * strip >= ncx) return;  // whole warp
  const int dof = P.bc != 0;
  const int I = 30 * strip + lane - 1;
  const int J0 = blockIdx.y * RB;
  f += (size_t)blockIdx.z * P.nx * P.ny;
  fc += (size_t)blockIdx.z * ncx * ncy;
  // the warp's window: columns 2(30 s - 1) + dof .. 2(30 s + 30) + dof + 1, rows 2 J0 + dof - 2 ..
  // 2 (J0 + RB) + dof, all strictly inside the grid (no boundary node, no outside node)
  const int x0 = 2 * (30 * strip - 1) + dof, x1 = 2 * (30 * strip + 30) + dof + 1;
  const int y0 = 2 * J0 + dof - 2, y1 = 2 * (J0 + RB) + dof;
  const bool interior = x0 >= 1 && x1 <= P.nx - 2 && y0 >= 1 && y1 <= P.ny - 2;
  if (interior) mg_down_band<T, true>(P, f, fc, ncx, ncy, omega, I, J0, RB, lane);
  else mg_down_band<T, false>(P, f, fc, ncx, ncy, omega, I, J0, RB, lane);
}

// y = (1 - omega) u + u0 + omega c S(u) / D [+ add], u = u0 + P ec, u0 = omega f / D: the fused
// bilinear correction and post-smoothing sweep.  Strip s, lane L: vertex columns 2V and 2V + 1
// with V = 30 s + L - 1 (vertex column v is grid column v - dof: Dirichlet grids hold interior
// unknowns, fine unknown g is vertex g + 1 and coarse unknown I is vertex I + 1, zero at the
// vertices the grid omits), so the lane needs coarse vertex V (the next lane supplies V + 1);
// outputs at lanes 1 .. 30.  Band: rows Y0 .. Y0 + RB - 1.
template <typename T, bool IN>
__device__ __forceinline__ void mg_up_band(const OpP<T>& P, const cx<T>* __restrict__ f, const cx<T>* __restrict__ ec,
                                           int ncx, int ncy, cx<T>* __restrict__ y, T omega,
                                           const cx<T>* __restrict__ add, int V, int Y0, int RB, int lane) {
  const int dof = P.bc != 0;
  const bool som = !IN && P.bc == 0;
  const T c4 = T(4) * P.c, c2H = P.c * T(2) * P.H, om1 = T(1) - omega, omc = omega * P.c;
  const int ga = 2 * V - dof, gb = ga + 1;
  const bool ain = IN || (ga >= 0 && ga < P.nx), bin = IN || (gb >= 0 && gb < P.nx);
  const int abnd = som && ain && (ga == 0 || ga == P.nx - 1), bbnd = som && bin && (gb == 0 || gb == P.nx - 1);
  const bool outl = lane >= 1 && lane <= 30;
  const int Ic = V - dof;
  const bool icin = Ic >= 0 && Ic < ncx;
  auto ecv = [&](int Jv) -> cx<T> {
    const int J = Jv - dof;
    return (icin && J >= 0 && J < ncy) ? ec[(size_t)J * ncx + Ic] : mk<T>(T(0), T(0));
  };
  const int ccol = max(min(ga, P.nx - 2), 0), fda = ga - ccol;
  auto load = [&](int gy, cx<T>& fa, cx<T>& fb, T& ka, T& kb) {
    if (IN) {
      const size_t o = (size_t)gy * P.nx + ga;
      fa = f[o];
      fb = f[o + 1];
      ka = P.k[o];
      kb = P.k[o + 1];
    } else {
      const bool rin = gy >= 0 && gy < P.ny;
      const size_t o = (size_t)max(gy, 0) * P.nx + ccol + fda;
      fa = (rin && ain) ? f[o] : mk<T>(T(0), T(0));
      fb = (rin && bin) ? f[o + 1] : mk<T>(T(0), T(0));
      ka = (rin && ain) ? P.k[o] : T(0);
      kb = (rin && bin) ? P.k[o + 1] : T(0);
    }
  };
  const int yb = Y0 - 1, ye = min(Y0 + RB, P.ny);  // window rows yb .. ye (inclusive)
  int gyv = yb + dof;
  int Jv = gyv >= 0 ? (gyv >> 1) : -((1 - gyv) >> 1);
  cx<T> c0 = ecv(Jv), c1 = ecv(Jv + 1), c2 = ecv(Jv + 2);  // coarse rows Jv .. Jv + 2 at column V
  cx<T> pfa[kPF], pfb[kPF];
  T pka[kPF], pkb[kPF];
#pragma unroll
  for (int q = 0; q < kPF; ++q) load(yb + q, pfa[q], pfb[q], pka[q], pkb[q]);
  cx<T> ua_m2 = mk<T>(T(0), T(0)), ub_m2 = ua_m2, ua_m1 = ua_m2, ub_m1 = ua_m2;
  cx<T> u0a_m1 = ua_m2, u0b_m1 = ua_m2;
  T dra_m1 = T(0), dia_m1 = T(0), iva_m1 = T(0), drb_m1 = T(0), dib_m1 = T(0), ivb_m1 = T(0);
  for (int y00 = yb; y00 <= ye; y00 += kPF) {
#pragma unroll
    for (int q = 0; q < kPF; ++q) {
      const int gy = y00 + q;
      if (gy > ye) break;
      const cx<T> fa = pfa[q], fb = pfb[q];
      const T ka = pka[q], kb = pkb[q];
      if (gy + kPF <= ye) load(gy + kPF, pfa[q], pfb[q], pka[q], pkb[q]);
      const int gv = gy + dof;
      const int Jn = gv >= 0 ? (gv >> 1) : -((1 - gv) >> 1);
      if (Jn != Jv) {  // advanced to the next coarse row
        Jv = Jn;
        c0 = c1;
        c1 = c2;
        c2 = ecv(Jv + 2);
      }
      // bilinear correction at vertex columns 2V (the coarse value) and 2V + 1 (with V + 1)
      const cx<T> cv = (gv & 1) ? T(0.5) * (c0 + c1) : c0;
      const cx<T> cn = mk<T>(__shfl_down_sync(0xffffffffu, cv.re, 1), __shfl_down_sync(0xffffffffu, cv.im, 1));
      const cx<T> ea = cv, eb = T(0.5) * (cv + cn);
      const bool rin = IN || (gy >= 0 && gy < P.ny);
      const int gyb = som && (gy == 0 || gy == P.ny - 1);
      cx<T> ua = mk<T>(T(0), T(0)), ub = ua, u0a = ua, u0b = ua;
      T dra = T(0), dia = T(0), iva = T(0), drb = T(0), dib = T(0), ivb = T(0);
      if (rin && ain) {
        const T k2 = ka * ka;
        dra = fma(-P.ksr, k2, c4);
        dia = -P.ksi * k2;
        if (som) {
          const int g = abnd + gyb;
          if (g) dia -= c2H * ka * T(g);
        }
        iva = r1_recip<T>(dra * dra + dia * dia);
        u0a = mk<T>(omega * (fa.re * dra + fa.im * dia) * iva, omega * (fa.im * dra - fa.re * dia) * iva);
        ua = u0a + ea;
      }
      if (rin && bin) {
        const T k2 = kb * kb;
        drb = fma(-P.ksr, k2, c4);
        dib = -P.ksi * k2;
        if (som) {
          const int g = bbnd + gyb;
          if (g) dib -= c2H * kb * T(g);
        }
        ivb = r1_recip<T>(drb * drb + dib * dib);
        u0b = mk<T>(omega * (fb.re * drb + fb.im * dib) * ivb, omega * (fb.im * drb - fb.re * dib) * ivb);
        ub = u0b + eb;
      }
      if (gy >= yb + 2) {  // output row gy - 1
        const int yr = gy - 1;
        cx<T> wa = mk<T>(__shfl_up_sync(0xffffffffu, ub_m1.re, 1), __shfl_up_sync(0xffffffffu, ub_m1.im, 1));
        cx<T> eb2 = mk<T>(__shfl_down_sync(0xffffffffu, ua_m1.re, 1), __shfl_down_sync(0xffffffffu, ua_m1.im, 1));
        cx<T> ea2 = ub_m1, wb = ua_m1;
        cx<T> sa = ua_m2, na = ua, sb = ub_m2, nb = ub;
        if (som) {
          if (ga == 0) wa = ea2;
          if (ga == P.nx - 1) ea2 = wa;
          if (gb == 0) wb = eb2;
          if (gb == P.nx - 1) eb2 = wb;
          if (yr == 0) {
            sa = na;
            sb = nb;
          }
          if (yr == P.ny - 1) {
            na = sa;
            nb = sb;
          }
        }
        if (outl && (IN || (yr >= Y0 && yr < P.ny))) {
          const size_t o = (size_t)yr * P.nx;
          if (ain) {
            const cx<T> sn = (wa + ea2) + (sa + na);
            const cx<T> qv = mk<T>((sn.re * dra_m1 + sn.im * dia_m1) * iva_m1, (sn.im * dra_m1 - sn.re * dia_m1) * iva_m1);
            cx<T> out = (om1 * ua_m1 + u0a_m1) + omc * qv;
            if (add) out = out + add[o + ga];
            y[o + ga] = out;
          }
          if (bin) {
            const cx<T> sn = (wb + eb2) + (sb + nb);
            const cx<T> qv = mk<T>((sn.re * drb_m1 + sn.im * dib_m1) * ivb_m1, (sn.im * drb_m1 - sn.re * dib_m1) * ivb_m1);
            cx<T> out = (om1 * ub_m1 + u0b_m1) + omc * qv;
            if (add) out = out + add[o + gb];
            y[o + gb] = out;
          }
        }
      }
      ua_m2 = ua_m1;
      ub_m2 = ub_m1;
      ua_m1 = ua;
      ub_m1 = ub;
      u0a_m1 = u0a;
      u0b_m1 = u0b;
      dra_m1 = dra;
      dia_m1 = dia;
      iva_m1 = iva;
      drb_m1 = drb;
      dib_m1 = dib;
      ivb_m1 = ivb;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_mg_up_r1(OpP<T> P, const cx<T>* __restrict__ f, const cx<T>* __restrict__ ec,
                                                  int ncx, int ncy, cx<T>* __restrict__ y, T omega,
                                                  const cx<T>* __restrict__ add, int RB) {
  P.k += (size_t)blockIdx.z * P.kstride;  // this right-hand side's wavenumber field
  const int lane = threadIdx.x & 31;
  const int strip = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int dof = P.bc != 0;
  if (60 * strip - dof >= P.nx) return;  // whole warp
  const int V = 30 * strip + lane - 1;
  const int Y0 = blockIdx.y * RB;
  const size_t off = (size_t)blockIdx.z * P.nx * P.ny;
  f += off;
  y += off;
  ec += (size_t)blockIdx.z * ncx * ncy;
  if (add) add += off;
  // window columns 60 s - 2 - dof .. 60 s + 59 - dof (lanes 0 .. 31), rows Y0 - 1 .. Y0 + RB: all
  // strictly inside the grid
  const int x0 = 60 * strip - 2 - dof, x1 = 60 * strip + 61 - dof;
  const bool interior = x0 >= 1 && x1 <= P.nx - 2 && Y0 - 1 >= 1 && Y0 + RB <= P.ny - 2;
  if (interior) mg_up_band<T, true>(P, f, ec, ncx, ncy, y, omega, add, V, Y0, RB, lane);
  else mg_up_band<T, false>(P, f, ec, ncx, ncy, y, omega, add, V, Y0, RB, lane);
}

template <typename T>
__global__ void __launch_bounds__(256) k_fw(const cx<T>* __restrict__ r, int nx, int ny, cx<T>* __restrict__ rc,
                                            int ncx, int ncy, int dof) {
  const size_t nc = (size_t)ncx * ncy;
  const size_t off = (size_t)blockIdx.y * nx * ny, offc = (size_t)blockIdx.y * nc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nc; i += (size_t)gridDim.x * blockDim.x) {
    int J = (int)(i / ncx), I = (int)(i - (size_t)J * ncx);
    cx<T> s = mk<T>(T(0), T(0));
    for (int b = -1; b <= 1; ++b) {
      int gy = 2 * J + b + dof;  // centred on fine 2J (2J + 1 on Dirichlet grids)
      if (gy < 0 || gy >= ny) continue;
      for (int a = -1; a <= 1; ++a) {
        int gx = 2 * I + a + dof;
        if (gx < 0 || gx >= nx) continue;
        T w = T((2 - (a < 0 ? -a : a)) * (2 - (b < 0 ? -b : b)));
        s = s + w * r[off + (size_t)gy * nx + gx];
      }
    }
    rc[offc + i] = T(0.0625) * s;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(const cx<T>* __restrict__ ec, int ncx, int ncy,
                                                     cx<T>* __restrict__ u, int nx, int ny, int dof) {
  const size_t n = (size_t)nx * ny;
  const size_t off = (size_t)blockIdx.y * n, offc = (size_t)blockIdx.y * ncx * ncy;
  // coarse value at vertex-grid coarse index (I, J); zero at the vertices a Dirichlet grid omits
  auto E = [&](int I, int J) -> cx<T> {
    I -= dof;
    J -= dof;
    return (I >= 0 && I < ncx && J >= 0 && J < ncy) ? ec[offc + (size_t)J * ncx + I] : mk<T>(T(0), T(0));
  };
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int gy = (int)(i / nx) + dof, gx = (int)(i % nx) + dof;
    int I = gx >> 1, J = gy >> 1, ex = gx & 1, ey = gy & 1;
    cx<T> a = E(I, J);
    if (ex) a = T(0.5) * (a + E(I + 1, J));
    if (ey) {
      cx<T> b = E(I, J + 1);
      if (ex) b = T(0.5) * (b + E(I + 1, J + 1));
      a = T(0.5) * (a + b);
    }
    u[off + i] = u[off + i] + a;
  }
}

// ---------------------------------------------------------------------------------------
template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return hz::ensure_dyn_smem(reinterpret_cast<const void*>(kernel), bytes);
}

inline unsigned grid1d(size_t n) {
  size_t b = (n + 255) / 256;
  size_t cap = 152 * 16;
  return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

template <typename T, typename TI, typename TO, int R>
cudaError_t level_op_r(hz::Ctx& c, const hz::OpDesc& d, int mode, const void* x, const void* f, void* y,
                       double omega, int nrhs) {
  OpP<T> P = make_op<T>(d);
  dim3 grid((d.nx + OXT - 1) / OXT, (d.ny + OYT - 1) / OYT, nrhs), block(BX, BY);
  size_t sm = tile_smem_bytes<T, R>(OXT, OYT);
  auto X = reinterpret_cast<const cx<TI>*>(x);
  auto F = reinterpret_cast<const cx<TI>*>(f);
  auto Y = reinterpret_cast<cx<TO>*>(y);
  cudaError_t e;
  double bytes = (double)nrhs * d.n() * (sizeof(cx<TI>) * (mode ? 2 : 1) + sizeof(cx<TO>) + sizeof(T));
  hz::ProfScope ps(c, hz::F_LEVEL_OP, bytes);
  if (mode == 0) {
    if ((e = set_smem(k_level_op<T, TI, TO, R, 0>, sm)) != cudaSuccess) return e;
    k_level_op<T, TI, TO, R, 0><<<grid, block, sm, c.s>>>(P, X, F, Y, T(omega));
  } else if (mode == 1) {
    if ((e = set_smem(k_level_op<T, TI, TO, R, 1>, sm)) != cudaSuccess) return e;
    k_level_op<T, TI, TO, R, 1><<<grid, block, sm, c.s>>>(P, X, F, Y, T(omega));
  } else {
    if ((e = set_smem(k_level_op<T, TI, TO, R, 2>, sm)) != cudaSuccess) return e;
    k_level_op<T, TI, TO, R, 2><<<grid, block, sm, c.s>>>(P, X, F, Y, T(omega));
  }
  return cudaGetLastError();
}

template <typename T, typename TI, typename TO>
cudaError_t level_op_t(hz::Ctx& c, const hz::OpDesc& d, int mode, const void* x, const void* f, void* y,
                       double omega, int nrhs) {
  switch (d.R) {
    case 1: return level_op_r<T, TI, TO, 1>(c, d, mode, x, f, y, omega, nrhs);
    case 2: return level_op_r<T, TI, TO, 2>(c, d, mode, x, f, y, omega, nrhs);
    case 3: return level_op_r<T, TI, TO, 3>(c, d, mode, x, f, y, omega, nrhs);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

namespace hz {

cudaError_t launch_level_op(Ctx& c, const OpDesc& op, int mode, int tcomp, int tx, int ty, const void* x,
                            const void* f, void* y, double omega, int nrhs) {
  if (tcomp == C128 && tx == C128 && ty == C128) return level_op_t<double, double, double>(c, op, mode, x, f, y, omega, nrhs);
  if (tcomp == C64 && tx == C64 && ty == C64) return level_op_t<float, float, float>(c, op, mode, x, f, y, omega, nrhs);
  if (tcomp == C128 && tx == C64 && ty == C128) return level_op_t<double, float, double>(c, op, mode, x, f, y, omega, nrhs);
  return cudaErrorInvalidValue;
}

template <typename T, int R>
static cudaError_t jz_r(Ctx& c, const OpDesc& d, const void* f, void* y, double omega, int nrhs) {
  ProfScope ps(c, F_MG_DOWN, (double)nrhs * d.n() * (2 * sizeof(cx<T>) + sizeof(T)));
  k_jacobi_zero<T, R><<<dim3(grid1d(d.n()), nrhs), 256, 0, c.s>>>(make_op<T>(d), reinterpret_cast<const cx<T>*>(f),
                                                                   reinterpret_cast<cx<T>*>(y), T(omega));
  return cudaGetLastError();
}

cudaError_t launch_jacobi_zero(Ctx& c, const OpDesc& op, int dt, const void* f, void* y, double omega, int nrhs) {
  if (dt == C128) {
    switch (op.R) {
      case 1: return jz_r<double, 1>(c, op, f, y, omega, nrhs);
      case 2: return jz_r<double, 2>(c, op, f, y, omega, nrhs);
      case 3: return jz_r<double, 3>(c, op, f, y, omega, nrhs);
    }
  } else {
    switch (op.R) {
      case 1: return jz_r<float, 1>(c, op, f, y, omega, nrhs);
      case 2: return jz_r<float, 2>(c, op, f, y, omega, nrhs);
      case 3: return jz_r<float, 3>(c, op, f, y, omega, nrhs);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T, typename TV, int R>
static cudaError_t dpr_r(Ctx& c, const OpDesc& d, const void* vtil, int ncx, int ncy, const void* v, void* t,
                         void* rtil, int nrhs) {
  OpP<T> P = make_op<T>(d);
  dim3 grid((d.nx + OXT - 1) / OXT, (d.ny + OYT - 1) / OYT, nrhs), block(BX, BY);
  const int CW = (OXT + 2 * R + 6) / 2 + 2, CH = (OYT + 2 * R + 6) / 2 + 2;
  size_t sm = tile_smem_bytes<T, R>(OXT, OYT) + sizeof(cx<T>) * (CW * CH + CH * (OXT + 2 * R));
  cudaError_t e = set_smem(k_defl_prolong_resid<T, TV, R>, sm);
  if (e != cudaSuccess) return e;
  double bytes = (double)nrhs * d.n() * (sizeof(cx<TV>) + sizeof(cx<T>) * (t ? 2 : 1) + sizeof(T) + sizeof(cx<T>) / 4.0);
  ProfScope ps(c, F_DEFL_PROLONG, bytes);
  k_defl_prolong_resid<T, TV, R><<<grid, block, sm, c.s>>>(P, reinterpret_cast<const cx<T>*>(vtil), ncx, ncy,
                                                           reinterpret_cast<const cx<TV>*>(v),
                                                           reinterpret_cast<cx<T>*>(t), reinterpret_cast<cx<T>*>(rtil));
  return cudaGetLastError();
}

template <typename T, typename TV>
static cudaError_t dpr_t(Ctx& c, const OpDesc& d, const void* vtil, int ncx, int ncy, const void* v, void* t,
                         void* rtil, int nrhs) {
  switch (d.R) {
    case 1: return dpr_r<T, TV, 1>(c, d, vtil, ncx, ncy, v, t, rtil, nrhs);
    case 2: return dpr_r<T, TV, 2>(c, d, vtil, ncx, ncy, v, t, rtil, nrhs);
    case 3: return dpr_r<T, TV, 3>(c, d, vtil, ncx, ncy, v, t, rtil, nrhs);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_defl_prolong_resid(Ctx& c, const OpDesc& op, int tcomp, int tv, const void* vtil, int ncx,
                                      int ncy, const void* v, void* t, void* rtil, int nrhs) {
  if (tcomp == C128 && tv == C128) return dpr_t<double, double>(c, op, vtil, ncx, ncy, v, t, rtil, nrhs);
  if (tcomp == C64 && tv == C64) return dpr_t<float, float>(c, op, vtil, ncx, ncy, v, t, rtil, nrhs);
  if (tcomp == C64 && tv == C128) return dpr_t<float, double>(c, op, vtil, ncx, ncy, v, t, rtil, nrhs);
  return cudaErrorInvalidValue;
}

cudaError_t launch_defl_prolong(Ctx& c, int dt, int nx, int ny, const void* w, void* t, int nrhs, int bc) {
  const int dof = bc != 0;
  int ncx = coarse_n(nx, bc), ncy = coarse_n(ny, bc);
  size_t n = (size_t)nx * ny;
  ProfScope ps(c, F_DEFL_PROLONG, (double)nrhs * n * elem_bytes(dt) * 1.25);
  if (dt == C128)
    k_defl_prolong<double><<<dim3(grid1d(n), nrhs), 256, 0, c.s>>>(reinterpret_cast<const cx<double>*>(w), ncx, ncy,
                                                                    reinterpret_cast<cx<double>*>(t), nx, ny, dof);
  else
    k_defl_prolong<float><<<dim3(grid1d(n), nrhs), 256, 0, c.s>>>(reinterpret_cast<const cx<float>*>(w), ncx, ncy,
                                                                   reinterpret_cast<cx<float>*>(t), nx, ny, dof);
  return cudaGetLastError();
}

template <typename TI, typename T>
static cudaError_t dr_t(Ctx& c, int nx, int ny, const void* v, void* vhat, int nrhs, int bc) {
  int ncx = coarse_n(nx, bc), ncy = coarse_n(ny, bc);
  constexpr int FW = 2 * RXC + 3, FH = 2 * RYC + 3;
  size_t sm = sizeof(cx<T>) * (FW * FH + FH * RXC);
  cudaError_t e = set_smem(k_defl_restrict<TI, T>, sm);
  if (e != cudaSuccess) return e;
  ProfScope ps(c, F_DEFL_RESTRICT, (double)nrhs * ((double)nx * ny * sizeof(cx<TI>) + (double)ncx * ncy * sizeof(cx<T>)));
  dim3 grid((ncx + RXC - 1) / RXC, (ncy + RYC - 1) / RYC, nrhs);
  k_defl_restrict<TI, T><<<grid, dim3(BX, BY), sm, c.s>>>(reinterpret_cast<const cx<TI>*>(v), nx, ny,
                                                          reinterpret_cast<cx<T>*>(vhat), ncx, ncy, bc != 0);
  return cudaGetLastError();
}

cudaError_t launch_defl_restrict(Ctx& c, int tin, int tout, int nx, int ny, const void* v, void* vhat, int nrhs,
                                 int bc) {
  if (tin == C128 && tout == C128) return dr_t<double, double>(c, nx, ny, v, vhat, nrhs, bc);
  if (tin == C64 && tout == C64) return dr_t<float, float>(c, nx, ny, v, vhat, nrhs, bc);
  if (tin == C128 && tout == C64) return dr_t<double, float>(c, nx, ny, v, vhat, nrhs, bc);
  return cudaErrorInvalidValue;
}

// Band height (rows per warp) of a strip sweep: the tallest band up to maxrb that still gives
// about 16 warps per SM (152 SMs), at least 2 rows.
static int band_rows(int strips, int rows, int nrhs, int maxrb) {
  const long long want = 152LL * 16;
  int rb = maxrb;
  while (rb > 2 && (long long)strips * ((rows + rb - 1) / rb) * nrhs < want) rb /= 2;
  return rb;
}

// Band heights of the strip sweeps chosen by timing (tune_mg_bands), per kernel, level shape and
// precision, process-wide; shapes never timed take band_rows.
std::mutex g_band_mu;
std::map<std::tuple<int, int, int, int>, int> g_band;
static int band_for(int kind, const OpDesc& d, int dt, int strips, int rows, int nrhs, int maxrb) {
  {
    std::lock_guard<std::mutex> lk(g_band_mu);
    auto it = g_band.find(std::make_tuple(kind, d.nx, d.ny, dt));
    if (it != g_band.end()) return it->second;
  }
  return band_rows(strips, rows, nrhs, maxrb);
}

template <typename T>
static void down_r1_rb(cudaStream_t s, const OpDesc& d, const void* f, void* fc, double omega, int nrhs, int RB) {
  const int ncx = coarse_n(d.nx, d.bc), ncy = coarse_n(d.ny, d.bc);
  const int strips = (ncx + 29) / 30;
  dim3 grid((strips + 7) / 8, (ncy + RB - 1) / RB, nrhs);
  k_mg_down_r1<T><<<grid, 256, 0, s>>>(make_op<T>(d), reinterpret_cast<const cx<T>*>(f), reinterpret_cast<cx<T>*>(fc),
                                       ncx, ncy, T(omega), RB);
}

template <typename T>
static void up_r1_rb(cudaStream_t s, const OpDesc& d, const void* f, const void* ec, void* y, double omega,
                     const void* add, int nrhs, int RB) {
  const int ncx = coarse_n(d.nx, d.bc), ncy = coarse_n(d.ny, d.bc);
  const int strips = (d.nx + d.bc + 59) / 60;
  dim3 grid((strips + 7) / 8, (d.ny + RB - 1) / RB, nrhs);
  k_mg_up_r1<T><<<grid, 256, 0, s>>>(make_op<T>(d), reinterpret_cast<const cx<T>*>(f),
                                     reinterpret_cast<const cx<T>*>(ec), ncx, ncy, reinterpret_cast<cx<T>*>(y), T(omega),
                                     reinterpret_cast<const cx<T>*>(add), RB);
}

template <typename T>
static cudaError_t down_r1(Ctx& c, const OpDesc& d, const void* f, void* fc, double omega, int nrhs) {
  const int ncx = coarse_n(d.nx, d.bc), ncy = coarse_n(d.ny, d.bc);
  ProfScope ps(c, F_MG_DOWN, (double)nrhs * ((double)d.n() * (sizeof(cx<T>) + sizeof(T)) + (double)ncx * ncy * sizeof(cx<T>)));
  const int RB = band_for(0, d, sizeof(T) == 8 ? C128 : C64, (ncx + 29) / 30, ncy, nrhs, 16);
  down_r1_rb<T>(c.s, d, f, fc, omega, nrhs, RB);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t up_r1(Ctx& c, const OpDesc& d, const void* f, const void* ec, void* y, double omega,
                         const void* add, int nrhs) {
  const int ncx = coarse_n(d.nx, d.bc), ncy = coarse_n(d.ny, d.bc);
  double bytes = (double)nrhs * ((double)d.n() * (sizeof(cx<T>) * (add ? 3 : 2) + sizeof(T)) + (double)ncx * ncy * sizeof(cx<T>));
  ProfScope ps(c, F_MG_UP, bytes);
  const int RB = band_for(1, d, sizeof(T) == 8 ? C128 : C64, (d.nx + d.bc + 59) / 60, d.ny, nrhs, 32);
  up_r1_rb<T>(c.s, d, f, ec, y, omega, add, nrhs, RB);
  return cudaGetLastError();
}

// Times both strip sweeps of one radius-1 multigrid level at every band height (twice, the
// second run counts) on the given buffers and keeps the fastest for this shape and precision.
template <typename T>
static cudaError_t tune_bands_t(Ctx& c, const OpDesc& d, const void* f, void* fc, const void* ec, void* y,
                                double omega, int nrhs) {
  static const int cand[] = {2, 4, 8, 16, 32};
  const int dt = sizeof(T) == 8 ? C128 : C64;
  {
    std::lock_guard<std::mutex> lk(g_band_mu);
    if (g_band.count(std::make_tuple(0, d.nx, d.ny, dt)) && g_band.count(std::make_tuple(1, d.nx, d.ny, dt)))
      return cudaSuccess;
  }
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  int best[2] = {0, 0};
  for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
    float tbest = 1e30f;
    for (int rb : cand) {
      float ms = 0;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, c.s);
        if (kind == 0) down_r1_rb<T>(c.s, d, f, fc, omega, nrhs, rb);
        else up_r1_rb<T>(c.s, d, f, ec, y, omega, nullptr, nrhs, rb);
        cudaEventRecord(e1, c.s);
        if ((e = cudaEventSynchronize(e1)) == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      }
      if (e == cudaSuccess && ms < tbest) {
        tbest = ms;
        best[kind] = rb;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_band_mu);
  g_band[std::make_tuple(0, d.nx, d.ny, dt)] = best[0];
  g_band[std::make_tuple(1, d.nx, d.ny, dt)] = best[1];
  return cudaGetLastError();
}

template <typename T, int R>
static cudaError_t down_r(Ctx& c, const OpDesc& d, const void* f, void* fc, double omega, int nrhs) {
  int ncx = coarse_n(d.nx, d.bc), ncy = coarse_n(d.ny, d.bc);
  constexpr int OX = 2 * DXC + 1, OY = 2 * DYC + 1;
  size_t sm = tile_smem_bytes<T, R>(OX, OY) + sizeof(cx<T>) * OX * OY;
  cudaError_t e = set_smem(k_mg_down<T, R>, sm);
  if (e != cudaSuccess) return e;
  ProfScope ps(c, F_MG_DOWN, (double)nrhs * ((double)d.n() * (sizeof(cx<T>) + sizeof(T)) + (double)ncx * ncy * sizeof(cx<T>)));
  dim3 grid((ncx + DXC - 1) / DXC, (ncy + DYC - 1) / DYC, nrhs);
  k_mg_down<T, R><<<grid, dim3(BX, BY), sm, c.s>>>(make_op<T>(d), reinterpret_cast<const cx<T>*>(f),
                                                   reinterpret_cast<cx<T>*>(fc), ncx, ncy, T(omega));
  return cudaGetLastError();
}

cudaError_t launch_mg_down(Ctx& c, const OpDesc& op, int dt, const void* f, void* fc, double omega, int nrhs) {
  if (dt == C128) {
    if (op.R == 1) return down_r1<double>(c, op, f, fc, omega, nrhs);
    if (op.R == 2) return down_r<double, 2>(c, op, f, fc, omega, nrhs);
    if (op.R == 3) return down_r<double, 3>(c, op, f, fc, omega, nrhs);
  } else {
    if (op.R == 1) return down_r1<float>(c, op, f, fc, omega, nrhs);
    if (op.R == 2) return down_r<float, 2>(c, op, f, fc, omega, nrhs);
    if (op.R == 3) return down_r<float, 3>(c, op, f, fc, omega, nrhs);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int R>
static cudaError_t up_r(Ctx& c, const OpDesc& d, const void* f, const void* ec, void* y, double omega,
                        const void* add, int nrhs) {
  int ncx = coarse_n(d.nx, d.bc), ncy = coarse_n(d.ny, d.bc);
  const int EW = (OXT + 2 * R) / 2 + 3, EH = (OYT + 2 * R) / 2 + 3;
  size_t sm = tile_smem_bytes<T, R>(OXT, OYT) + sizeof(cx<T>) * EW * EH;
  cudaError_t e = set_smem(k_mg_up<T, R>, sm);
  if (e != cudaSuccess) return e;
  double bytes = (double)nrhs * ((double)d.n() * (sizeof(cx<T>) * (add ? 3 : 2) + sizeof(T)) + (double)ncx * ncy * sizeof(cx<T>));
  ProfScope ps(c, F_MG_UP, bytes);
  dim3 grid((d.nx + OXT - 1) / OXT, (d.ny + OYT - 1) / OYT, nrhs);
  k_mg_up<T, R><<<grid, dim3(BX, BY), sm, c.s>>>(make_op<T>(d), reinterpret_cast<const cx<T>*>(f),
                                                 reinterpret_cast<const cx<T>*>(ec), ncx, ncy,
                                                 reinterpret_cast<cx<T>*>(y), T(omega),
                                                 reinterpret_cast<const cx<T>*>(add));
  return cudaGetLastError();
}

cudaError_t launch_mg_up(Ctx& c, const OpDesc& op, int dt, const void* f, const void* ec, void* y, double omega,
                         const void* add, int tadd, void* yout2, int tout2, int nrhs) {
  (void)tadd;
  (void)yout2;
  (void)tout2;
  if (dt == C128) {
    if (op.R == 1) return up_r1<double>(c, op, f, ec, y, omega, add, nrhs);
    if (op.R == 2) return up_r<double, 2>(c, op, f, ec, y, omega, add, nrhs);
    if (op.R == 3) return up_r<double, 3>(c, op, f, ec, y, omega, add, nrhs);
  } else {
    if (op.R == 1) return up_r1<float>(c, op, f, ec, y, omega, add, nrhs);
    if (op.R == 2) return up_r<float, 2>(c, op, f, ec, y, omega, add, nrhs);
    if (op.R == 3) return up_r<float, 3>(c, op, f, ec, y, omega, add, nrhs);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tune_mg_bands(Ctx& c, const OpDesc& op, int dt, const void* f, void* fc, const void* ec, void* y,
                          double omega, int nrhs) {
  if (op.R != 1) return cudaSuccess;  // only the radius-1 strip sweeps have a band shape
  if (dt == C128) return tune_bands_t<double>(c, op, f, fc, ec, y, omega, nrhs);
  return tune_bands_t<float>(c, op, f, fc, ec, y, omega, nrhs);
}

int mg_band_rows(int kind, int nx, int ny, int dt) {
  std::lock_guard<std::mutex> lk(g_band_mu);
  auto it = g_band.find(std::make_tuple(kind, nx, ny, dt));
  return it == g_band.end() ? 0 : it->second;
}

cudaError_t launch_fw(Ctx& c, int dt, int nx, int ny, const void* r, void* rc, int nrhs, int bc) {
  const int dof = bc != 0;
  int ncx = coarse_n(nx, bc), ncy = coarse_n(ny, bc);
  size_t nc = (size_t)ncx * ncy;
  ProfScope ps(c, F_MISC, (double)nrhs * ((double)nx * ny + nc) * elem_bytes(dt));
  if (dt == C128)
    k_fw<double><<<dim3(grid1d(nc), nrhs), 256, 0, c.s>>>(reinterpret_cast<const cx<double>*>(r), nx, ny,
                                                           reinterpret_cast<cx<double>*>(rc), ncx, ncy, dof);
  else
    k_fw<float><<<dim3(grid1d(nc), nrhs), 256, 0, c.s>>>(reinterpret_cast<const cx<float>*>(r), nx, ny,
                                                          reinterpret_cast<cx<float>*>(rc), ncx, ncy, dof);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(Ctx& c, int dt, int nx, int ny, const void* ec, void* u, int nrhs, int bc) {
  const int dof = bc != 0;
  int ncx = coarse_n(nx, bc), ncy = coarse_n(ny, bc);
  size_t n = (size_t)nx * ny;
  ProfScope ps(c, F_MISC, (double)nrhs * (2.0 * n + (double)ncx * ncy) * elem_bytes(dt));
  if (dt == C128)
    k_prolong_add<double><<<dim3(grid1d(n), nrhs), 256, 0, c.s>>>(reinterpret_cast<const cx<double>*>(ec), ncx, ncy,
                                                                   reinterpret_cast<cx<double>*>(u), nx, ny, dof);
  else
    k_prolong_add<float><<<dim3(grid1d(n), nrhs), 256, 0, c.s>>>(reinterpret_cast<const cx<float>*>(ec), ncx, ncy,
                                                                  reinterpret_cast<cx<float>*>(u), nx, ny, dof);
  return cudaGetLastError();
}

}  // namespace hz
