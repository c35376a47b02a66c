// Device-side building blocks shared by the stencil kernels.
//
// Layout: one level vector is ny rows of nx interleaved complex values (x fastest);
// a batch of nrhs vectors is contiguous with stride nx*ny.  blockIdx.z selects the rhs.
//
// Tile engine.  A CTA owns an output window of the grid.  It stages the input field,
// extended by the stencil radius R, in shared memory, fills the Sommerfeld ghost layer
// (u_ghost = u_inner + 2 H i k_boundary u_boundary, Section 2.1), and evaluates the
// level operator at each output node:
//   R = 1 : the 5-point rows of Section 2.1 (ghosts already substituted in the tile);
//   R >= 2: the separable Galerkin stencil of Section 3.3 at interior nodes,
//           Lap = c (L_y M_x + M_y L_x) u,  K = M_y M_x (k^2 u),  out = Lap - sigma K,
//           computed as three x-passes and two y-passes; physical-boundary nodes use
//           the 5-point row at the level spacing (Section 3.3, "Boundary").
// Cells of the extended tile outside the grid are zero except the first ghost layer
// (one coordinate outside by exactly one); ghost wavenumbers are zero, so the
// wavenumber part sees zeros outside the grid.  Homogeneous Dirichlet grids (bc = 1,
// interior unknowns only) have no ghost layer and no boundary rows: the level's stencil
// applies at every node with zeros outside.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hzd {

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T r, T i) {
  cx<T> z;
  z.re = r;
  z.im = i;
  return z;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk<T>(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk<T>(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk<T>(s * a.re, s * a.im); }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// a / b for complex b
template <typename T>
__device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b) {
  T d = b.re * b.re + b.im * b.im;
  T inv = T(1) / d;
  return mk<T>((a.re * b.re + a.im * b.im) * inv, (a.im * b.re - a.re * b.im) * inv);
}
template <typename TO, typename TI>
__device__ __forceinline__ cx<TO> cvt(cx<TI> a) {
  return mk<TO>(TO(a.re), TO(a.im));
}

// Operator of one grid (a deflation level or a multigrid level).
//   R == 1 : out = c (4 u - sum of 4 neighbours) - sigma * ks * k^2 u
//   R >= 2 : interior out = c (L (x) M + M (x) L) u - sigma (M (x) M)(k^2 u), boundary as R == 1
// sigma = 1 for A, beta1 + i beta2 for the CSLP M.  ks = 4^(l-1) (Galerkin scale).
template <typename T>
struct OpP {
  int nx, ny;
  int R;            // stencil radius (also a template parameter of the kernels)
  int bc;           // 0 Sommerfeld, 1 Dirichlet
  int srow;         // 1: boundary rows scaled by 1/2 per boundary side (symmetric form)
  T c;              // Laplacian scale
  T H;              // ghost spacing (2 H i k)
  T ks;             // wavenumber-stencil sum
  T sr, si;         // sigma
  T ksr, ksi;       // ks * sigma
  T m[7], l[7];     // 1-D masks, index d + R (R >= 2)
  const T* k;       // wavenumber, nx*ny
  size_t kstride;   // elements between the wavenumber fields of consecutive right-hand sides
                    // (0: one field shared by the batch); kernels offset k by their rhs index
};

// Physical boundary sides a node touches.  Dirichlet grids hold interior unknowns only, so
// none of their nodes takes a boundary row: every node uses the level's stencil, zero outside.
template <typename T>
__device__ __forceinline__ int bsides(const OpP<T>& P, int gx, int gy) {
  if (P.bc != 0) return 0;
  return (gx == 0) + (gx == P.nx - 1) + (gy == 0) + (gy == P.ny - 1);
}

// Exact diagonal of the operator at an in-grid node (matches the ghost substitution).
template <typename T, int R>
__device__ __forceinline__ cx<T> op_diag(const OpP<T>& P, int gx, int gy) {
  T k = P.k[(size_t)gy * P.nx + gx];
  T k2 = k * k;
  int g = bsides(P, gx, gy);
  if (R == 1 || g > 0) {
    T dre = T(4) * P.c - P.sr * P.ks * k2;
    T dim = -P.si * P.ks * k2;
    if (P.bc == 0) dim -= P.c * T(2) * P.H * k * T(g);
    return mk<T>(dre, dim);
  } else {
    T lap = P.c * T(2) * P.l[R] * P.m[R];
    if (P.bc == 0) {  // a Sommerfeld ghost two steps away holds this node with coefficient 1
      T extra = P.c * (P.l[R] * P.m[R + 2] + P.m[R] * P.l[R + 2]);
      int near = (gx == 1) + (gx == P.nx - 2) + (gy == 1) + (gy == P.ny - 2);
      lap += extra * T(near);
    }
    T kc = P.m[R] * P.m[R] * k2;
    return mk<T>(lap - P.sr * kc, -P.si * kc);
  }
}

// Shared-memory tile: output window OX x OY at grid origin (ox0, oy0), extended by R.
template <typename T, int R>
struct TileView {
  cx<T>* U;      // (OY + 2R) x (OX + 2R): field with ghost layer
  cx<T>* W;      // same shape: k^2 * field inside the grid, 0 outside (R >= 2 only)
  cx<T>* XA;     // (OY + 2R) x OX : L_x U      (R >= 2 only)
  cx<T>* XB;     //                  M_x U
  cx<T>* XC;     //                  M_x W
  int OX, OY, ox0, oy0;
  __device__ __forceinline__ int WX() const { return OX + 2 * R; }
  __device__ __forceinline__ int WY() const { return OY + 2 * R; }
  __device__ __forceinline__ cx<T>& u(int cx_, int cy_) const { return U[cy_ * WX() + cx_]; }
};

template <typename T, int R>
__host__ __device__ constexpr size_t tile_smem_bytes(int OX, int OY) {
  return sizeof(cx<T>) * ((size_t)(OY + 2 * R) * (OX + 2 * R) * (R >= 2 ? 2 : 1) +
                          (R >= 2 ? (size_t)3 * (OY + 2 * R) * OX : 0));
}

template <typename T, int R>
__device__ __forceinline__ TileView<T, R> make_tile(void* smem, int OX, int OY, int ox0, int oy0) {
  TileView<T, R> t;
  t.OX = OX;
  t.OY = OY;
  t.ox0 = ox0;
  t.oy0 = oy0;
  cx<T>* p = reinterpret_cast<cx<T>*>(smem);
  size_t wsz = (size_t)(OY + 2 * R) * (OX + 2 * R);
  t.U = p;
  p += wsz;
  if (R >= 2) {
    t.W = p;
    p += wsz;
    t.XA = p;
    p += (size_t)(OY + 2 * R) * OX;
    t.XB = p;
    p += (size_t)(OY + 2 * R) * OX;
    t.XC = p;
  } else {
    t.W = t.XA = t.XB = t.XC = nullptr;
  }
  return t;
}

template <typename T, int R>
__device__ __forceinline__ void tile_finish(const TileView<T, R>& t, const OpP<T>& P);

// Stage 1: fill in-grid cells from src(gx, gy) (out-of-grid cells = 0) and W = k^2 u.
// Stage 2: Sommerfeld ghost layer.  Stage 3 (R >= 2): x-passes.  Ends synchronised.
template <typename T, int R, class Src>
__device__ __forceinline__ void tile_fill(const TileView<T, R>& t, const OpP<T>& P, const Src& src) {
  const int WX = t.WX(), WY = t.WY();
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int gx0 = t.ox0 - R, gy0 = t.oy0 - R;
  for (int idx = tid; idx < WX * WY; idx += nthr) {
    int cy = idx / WX, cxx = idx - cy * WX;
    int gx = gx0 + cxx, gy = gy0 + cy;
    cx<T> v = mk<T>(T(0), T(0));
    cx<T> w = v;
    if (gx >= 0 && gx < P.nx && gy >= 0 && gy < P.ny) {
      v = src(gx, gy);
      if (R >= 2) {
        T k = P.k[(size_t)gy * P.nx + gx];
        w = (k * k) * v;
      }
    }
    t.U[idx] = v;
    if (R >= 2) t.W[idx] = w;
  }
  __syncthreads();
  tile_finish<T, R>(t, P);
}

// Stages 2 and 3 of tile_fill (ghost layer, x-passes) on a tile whose U (and W) are staged
// and synchronised.  Ends synchronised.
template <typename T, int R>
__device__ __forceinline__ void tile_finish(const TileView<T, R>& t, const OpP<T>& P) {
  const int WX = t.WX(), WY = t.WY();
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int gx0 = t.ox0 - R, gy0 = t.oy0 - R;
  if (P.bc == 0) {
    const T two_h = T(2) * P.H;
    // left (gx = -1) and right (gx = nx) ghost columns, rows inside the grid
    const int cl = -1 - gx0, cr = P.nx - gx0;
    for (int cy = tid; cy < WY; cy += nthr) {
      int gy = gy0 + cy;
      if (gy < 0 || gy >= P.ny) continue;
      if (cl >= 0 && cl < WX) {
        T k = P.k[(size_t)gy * P.nx + 0];
        cx<T> ub = t.U[cy * WX + cl + 1], ui = t.U[cy * WX + cl + 2];
        t.U[cy * WX + cl] = mk<T>(ui.re - two_h * k * ub.im, ui.im + two_h * k * ub.re);
      }
      if (cr >= 0 && cr < WX) {
        T k = P.k[(size_t)gy * P.nx + P.nx - 1];
        cx<T> ub = t.U[cy * WX + cr - 1], ui = t.U[cy * WX + cr - 2];
        t.U[cy * WX + cr] = mk<T>(ui.re - two_h * k * ub.im, ui.im + two_h * k * ub.re);
      }
    }
    const int rb = -1 - gy0, rt = P.ny - gy0;
    for (int cxx = tid; cxx < WX; cxx += nthr) {
      int gx = gx0 + cxx;
      if (gx < 0 || gx >= P.nx) continue;
      if (rb >= 0 && rb < WY) {
        T k = P.k[gx];
        cx<T> ub = t.U[(rb + 1) * WX + cxx], ui = t.U[(rb + 2) * WX + cxx];
        t.U[rb * WX + cxx] = mk<T>(ui.re - two_h * k * ub.im, ui.im + two_h * k * ub.re);
      }
      if (rt >= 0 && rt < WY) {
        T k = P.k[(size_t)(P.ny - 1) * P.nx + gx];
        cx<T> ub = t.U[(rt - 1) * WX + cxx], ui = t.U[(rt - 2) * WX + cxx];
        t.U[rt * WX + cxx] = mk<T>(ui.re - two_h * k * ub.im, ui.im + two_h * k * ub.re);
      }
    }
    __syncthreads();
  }
  if (R >= 2) {
    // x-passes with register windows: each work item is one tile row and 4 consecutive
    // output columns, computed from 4 + 2R staged values per field
    const int OX = t.OX;
    const int nseg = (OX + 3) / 4;
    for (int it = tid; it < WY * nseg; it += nthr) {
      const int cy = it / nseg, sx = (it - cy * nseg) * 4;
      const cx<T>* ur = t.U + cy * WX + sx;
      const cx<T>* wr = t.W + cy * WX + sx;
      cx<T> u[4 + 2 * R], w[4 + 2 * R];
#pragma unroll
      for (int k = 0; k < 4 + 2 * R; ++k) {
        const bool ok = sx + k < WX;
        u[k] = ok ? ur[k] : mk<T>(T(0), T(0));
        w[k] = ok ? wr[k] : mk<T>(T(0), T(0));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (sx + q >= OX) break;
        cx<T> a = mk<T>(T(0), T(0)), b = a, c = a;
#pragma unroll
        for (int d = 0; d <= 2 * R; ++d) {
          a = a + P.l[d] * u[q + d];
          b = b + P.m[d] * u[q + d];
          c = c + P.m[d] * w[q + d];
        }
        const int o = cy * OX + sx + q;
        t.XA[o] = a;
        t.XB[o] = b;
        t.XC[o] = c;
      }
    }
    __syncthreads();
  }
}

// Operator value at output cell (ox, oy) of the tile (grid node ox0 + ox, oy0 + oy).
template <typename T, int R>
__device__ __forceinline__ cx<T> tile_op(const TileView<T, R>& t, const OpP<T>& P, int ox, int oy) {
  const int WX = t.WX();
  const int gx = t.ox0 + ox, gy = t.oy0 + oy;
  const cx<T>* uc = t.U + (oy + R) * WX + (ox + R);
  if (R == 1 || bsides(P, gx, gy) > 0) {
    // c (4 u - s) - sigma ks k^2 u = (4c - sr ks k^2) u - i si ks k^2 u - c s
    const cx<T> s = (uc[1] + uc[-1]) + (uc[WX] + uc[-WX]);
    const T k = P.k[(size_t)gy * P.nx + gx];
    const T k2 = k * k;
    const T dr = fma(-P.ksr, k2, T(4) * P.c);
    const T di = P.ksi * k2;
    const cx<T> u = *uc;
    cx<T> v = mk<T>(fma(dr, u.re, fma(di, u.im, -P.c * s.re)), fma(dr, u.im, fma(-di, u.re, -P.c * s.im)));
    if (P.srow) {
      const int g = bsides(P, gx, gy);
      if (g) v = (g == 1 ? T(0.5) : T(0.25)) * v;
    }
    return v;
  } else {
    const int OX = t.OX;
    cx<T> lap = mk<T>(T(0), T(0)), kk = lap;
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) {
      int row = (oy + d) * OX + ox;
      lap = lap + P.m[d] * t.XA[row];
      lap = lap + P.l[d] * t.XB[row];
      kk = kk + P.m[d] * t.XC[row];
    }
    return mk<T>(P.c * lap.re - (P.sr * kk.re - P.si * kk.im), P.c * lap.im - (P.sr * kk.im + P.si * kk.re));
  }
}

}  // namespace hzd

namespace hzd {

// Operator values at up to SEG vertically consecutive output cells (ox, oy0 + q), q < cnt.
// For R >= 2 the y-passes run on register windows of SEG + 2R staged rows per field; cells on
// the physical boundary take the 5-point row through tile_op.
template <typename T, int R, int SEG = 4>
__device__ __forceinline__ void tile_op_seg(const TileView<T, R>& t, const OpP<T>& P, int ox, int oy0, int cnt,
                                            cx<T> (&out)[4]) {
  if (R == 1) {
#pragma unroll
    for (int q = 0; q < SEG; ++q)
      if (q < cnt) out[q] = tile_op<T, R>(t, P, ox, oy0 + q);
    return;
  }
  const int OX = t.OX, WY = t.WY();
  cx<T> a[SEG + 2 * R], b[SEG + 2 * R], c[SEG + 2 * R];
#pragma unroll
  for (int k = 0; k < SEG + 2 * R; ++k) {
    const int row = oy0 + k;
    const bool ok = row < WY;
    const int o = row * OX + ox;
    a[k] = ok ? t.XA[o] : mk<T>(T(0), T(0));
    b[k] = ok ? t.XB[o] : mk<T>(T(0), T(0));
    c[k] = ok ? t.XC[o] : mk<T>(T(0), T(0));
  }
  const int gx = t.ox0 + ox;
#pragma unroll
  for (int q = 0; q < SEG; ++q) {
    if (q >= cnt) break;
    const int gy = t.oy0 + oy0 + q;
    if (bsides(P, gx, gy) > 0) {
      out[q] = tile_op<T, R>(t, P, ox, oy0 + q);
      continue;
    }
    cx<T> lap = mk<T>(T(0), T(0)), kk = lap;
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) {
      lap = lap + P.m[d] * a[q + d];
      lap = lap + P.l[d] * b[q + d];
      kk = kk + P.m[d] * c[q + d];
    }
    out[q] = mk<T>(P.c * lap.re - (P.sr * kk.re - P.si * kk.im), P.c * lap.im - (P.sr * kk.im + P.si * kk.re));
  }
}

}  // namespace hzd
