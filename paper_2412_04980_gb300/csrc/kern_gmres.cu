// Persistent GMRES for the CSLP inverse on the coarse levels (Section 4.2: unpreconditioned
// GMRES on M_l to relative tolerance 0.1, at most floor(6 N_l^(1/4)) iterations, zero
// initial guess).  One cooperative launch runs the whole solve:
//
//   op      w_new = M_l (s * w_old) by the shared tile engine; the owning tile also writes
//           V_j = s * w_old (normalisation fused into the stencil, w ping-pongs).
//   dots    h = V^H w and ||w||^2 over grid-stride slices, 8 vectors per pass.
//   update  w -= V h with ||w||^2; a second classical pass only when ||w'|| < ||w||/sqrt(2).
//   reduce  every CTA sums all CTA partials itself in one fixed order, so every CTA holds
//           bitwise-identical coefficients and takes identical decisions.
//   Givens  complex rotations and the residual estimate |g_{j+1}| in FP64, redundantly in
//           each CTA; CTA 0 keeps the rotated Hessenberg columns for the final solve.
//
// Two launch forms share the kernel body.  Cooperative grid (large levels): grid-wide
// ordering by a sense-reversal barrier whose spin is bounded by a clock64 budget (a CTA
// that runs out sets an error flag, every CTA returns at its next barrier, and the host
// reports HZ_ETIMEOUT); the last CTA to arrive reduces the partials.  Thread-block cluster
// (small levels, where a barrier costs more than the vector work): the whole solve runs in
// one cluster of up to 16 CTAs, ordered by the hardware cluster barrier (release/acquire at
// cluster scope), and every CTA sums the cluster's partials itself in one fixed order.
// Barriers separate every write of a partial buffer from the reads of its previous contents.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "hz_core.h"
#include "hz_device.cuh"

using namespace hzd;

namespace {

constexpr int NT = 512;
constexpr int NW = NT / 32;
constexpr int kWred = NW * 2 * 16 + NW;  // warp partials of up to 16 complex values, then NW norms
// Operator tiles of the grid form: TS = 0 -> 32 x 16 nodes, TS = 1 -> 64 x 32 (large FP32 levels,
// where fewer, fuller tiles per CTA cut the per-tile synchronisation; measured on GB300 at
// 1025^2: operator phase 28.7 -> 18.8 us per iteration).
template <int TS> struct TileShape { static constexpr int X = 32, Y = 16; };
template <> struct TileShape<1> { static constexpr int X = 64, Y = 32; };
constexpr long long kSpinCycles = 4000000000LL;  // ~2 s at 2 GHz per barrier wait

// Loads of data that other CTAs write during the launch bypass L1 (not coherent across SMs).
__device__ __forceinline__ cx<float> ldcg(const cx<float>* p) {
  float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return mk<float>(v.x, v.y);
}
__device__ __forceinline__ cx<double> ldcg(const cx<double>* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return mk<double>(v.x, v.y);
}

__device__ __forceinline__ bool failed(const hz::GmresState* gs) { return *((volatile const int*)&gs->err) != 0; }

// Asynchronous 8-byte global -> shared copies (one complex FP32 value; any 8-byte aligned source,
// so the odd-length vectors of 2^k + 1 grids need no padding).  A thread waits only for its own
// copies and reads only the slots it filled, so the pipelines below need no CTA barrier.
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The FP32 slice dots stream the basis through a ring of kStages stages of 8 x 512 complex values
// in shared memory (the operator tile's space, unused between operator phases).
constexpr int kStages = 3;
constexpr size_t kRingBytes = (size_t)kStages * 8 * 512 * 8;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Device-side timing of one launch (or one cluster's solve): CTA 0 stamps the entry time before
// the first barrier, the last CTA to finish adds the elapsed time to the totals.  Works inside
// CUDA graphs, where host-side event pairs cannot bracket the launch.
__device__ __forceinline__ void timing_begin(hz::GmresState* st, unsigned bid) {
  if (bid == 0 && threadIdx.x == 0) {
    st->t_start = gtimer();
    st->done = 0u;
  }
}
__device__ __forceinline__ void timing_end(hz::GmresState* st, unsigned G) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned d = atomicAdd(&st->done, 1u);
    if (d == G - 1) {
      __threadfence();
      const unsigned long long t0 = *((volatile unsigned long long*)&st->t_start);
      st->total_ns += (long long)(gtimer() - t0);
      st->launches += 1;
    }
  }
}

__device__ __forceinline__ bool grid_sync(hz::GmresState* gs, unsigned nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &gs->gen;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&gs->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&gs->count, 0u);
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (failed(gs)) break;
        if (clock64() - t0 > kSpinCycles) {
          atomicExch(&gs->err, 1);
          break;
        }
        __nanosleep(40);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return !failed(gs);
}

// Grid barrier that also reduces CTA partials: after the barrier every CTA sums
// part[i * nblocks + b] over all CTAs b for i < m itself (value-major, so the K lanes that
// share a value read consecutive CTAs' partials; then a fixed shuffle tree), so every CTA
// holds bitwise-identical sums in out[] (shared) without a serial reduction by one CTA and a
// second wait for it.
__device__ __forceinline__ bool grid_reduce(hz::GmresState* gs, unsigned nblocks, const double* part, int pstride,
                                            int m, double* /*red*/, double* out) {
  if (!grid_sync(gs, nblocks)) return false;
  int K = 32;
  while (K > 1 && (NT / K) < m) K >>= 1;
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / K;
  for (int base = 0; base < m; base += (NT / 32) * per_warp) {
    const int i = base + (threadIdx.x >> 5) * per_warp + lane / K;
    const int k = lane % K;
    double t = 0;
    if (i < m) {
      const double* pi = part + (size_t)i * nblocks;
      double a[16];
      int b = k;
      for (; b + 15 * K < (int)nblocks; b += 16 * K) {
#pragma unroll
        for (int u = 0; u < 16; ++u) a[u] = __ldcg(pi + b + u * K);
#pragma unroll
        for (int u = 0; u < 16; ++u) t += a[u];
      }
      for (; b < (int)nblocks; b += K) t += __ldcg(pi + b);
    }
    for (int o = K / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (i < m && k == 0) out[i] = t;
  }
  __syncthreads();
  return true;
}

// Hardware barrier over all threads of all CTAs of the cluster; orders global-memory writes
// before it with reads after it (release / acquire at cluster scope).
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <bool CL>
__device__ __forceinline__ bool bar_all(hz::GmresState* gs, unsigned nblocks) {
  if constexpr (CL) {
    cluster_barrier();
    return true;
  } else {
    return grid_sync(gs, nblocks);
  }
}

constexpr int kMaxCluster = 16;

// Barrier + reduction of the CTA partials part[i * nblocks + b], b < nblocks, i < m into out[]
// (shared).  Cluster form: every CTA adds the partials itself in increasing b, so all CTAs
// hold bitwise-identical sums.
template <bool CL>
__device__ __forceinline__ bool reduce_all(hz::GmresState* gs, unsigned nblocks, const double* part, int pstride,
                                           int m, double* red, double* out) {
  if constexpr (CL) {
    cluster_barrier();
    for (int i = threadIdx.x; i < m; i += NT) {
      double a[kMaxCluster];
#pragma unroll
      for (int b = 0; b < kMaxCluster; ++b) a[b] = b < (int)nblocks ? __ldcg(part + (size_t)i * nblocks + b) : 0.0;
      double t = a[0];
#pragma unroll
      for (int b = 1; b < kMaxCluster; ++b) t += a[b];
      out[i] = t;
    }
    __syncthreads();
    return true;
  } else {
    return grid_reduce(gs, nblocks, part, pstride, m, red, out);
  }
}

// Convert m reduced FP64 values to the arithmetic type in parallel and return, in every
// thread, the sum of squares of the first m2 of them (one warp reduction).
template <typename T>
__device__ __forceinline__ T typed_copy_sumsq(const double* h, T* hT, int m, int m2, T* sred) {
  for (int i = threadIdx.x; i < m; i += NT) hT[i] = T(h[i]);
  __syncthreads();
  if (threadIdx.x < 32) {
    T acc = T(0);
    for (int i = threadIdx.x; i < m2; i += 32) acc += hT[i] * hT[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) *sred = acc;
  }
  __syncthreads();
  return *sred;
}

// Warp transpose-reduction (see kern_vec.cu): lane l ends with the warp sum of value l % CNT.
template <typename T, int CNT>
__device__ __forceinline__ T warp_tsum(T (&v)[CNT]) {
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
  return x;
}

// Software-pipelined staging of the operator tiles: every thread holds the source values (and
// wavenumbers) of up to PF cells of the next tile in registers while the current tile computes.
template <typename T, int R, int TOX, int TOY>
struct TilePrefetch {
  static constexpr int PF = ((TOX + 2 * R) * (TOY + 2 * R) + NT - 1) / NT;
  cx<T> v[PF];
  T k[PF];
  __device__ __forceinline__ void load(const OpP<T>& P, const cx<T>* src, int ox0, int oy0) {
    constexpr int WX = TOX + 2 * R, WY = TOY + 2 * R;
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int idx = threadIdx.x + u * NT;
      const int cy = idx / WX, cxx = idx - cy * WX;
      const int gx = ox0 - R + cxx, gy = oy0 - R + cy;
      const bool in = idx < WX * WY && gx >= 0 && gx < P.nx && gy >= 0 && gy < P.ny;
      v[u] = in ? ldcg(src + (size_t)gy * P.nx + gx) : mk<T>(T(0), T(0));
      if (R >= 2) k[u] = in ? P.k[(size_t)gy * P.nx + gx] : T(0);
    }
  }
  // U = s v (zero outside the grid), W = k^2 U
  __device__ __forceinline__ void store(const TileView<T, R>& t, T s) const {
    constexpr int WX = TOX + 2 * R, WY = TOY + 2 * R;
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int idx = threadIdx.x + u * NT;
      if (idx < WX * WY) {
        const cx<T> sv = s * v[u];
        t.U[idx] = sv;
        if (R >= 2) t.W[idx] = (k[u] * k[u]) * sv;
      }
    }
  }
};

struct KShared {  // Krylov scratch in shared memory (after the tile)
  double* h;      // 2 * (cap + 1) + 1 reduced values of the current pass
  double* h1;     // first-pass coefficients kept for the Hessenberg column
  double* gc;     // cap Givens cosines
  double* gs;     // 2 * cap Givens sines (complex)
  double* g;      // 2 * (cap + 1) rotated right-hand side
  double* wred;   // NW warps x 16 values, then NW norms
  int* flags;     // [0] stop, [1] reorth
  double* scal;   // [0] next scale, [1] beta, [2] ||w||^2, [3] ||w'||^2
};

// Contiguous slice of the vector owned by CTA bid of the G CTAs that share one solve.
__device__ __forceinline__ void my_slice(size_t n, unsigned bid, unsigned G, size_t& s0, size_t& s1) {
  const size_t S = (n + G - 1) / G;
  s0 = (size_t)bid * S;
  s1 = s0 + S < n ? s0 + S : n;
  if (s0 > n) s0 = n;
}

// CTA partials of h_i = V_i^H w (i < nv) and, with with_norm, ||w||^2 over this CTA's slice.
// Warps split the vectors (warp q takes i = q, q + NW, ...; the norm is one more "vector"),
// lanes stream the slice; every partial is a complete sum over the slice, written by one lane.
template <typename T>
__device__ void dots_warp(const cx<T>* V, size_t n, int nv, const cx<T>* w, double* part, int pstride, bool with_norm,
                          unsigned bid, unsigned G) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  size_t s0, s1;
  my_slice(n, bid, G, s0, s1);
  const int jobs = nv + (with_norm ? 1 : 0);
  for (int i = wid; i < jobs; i += NW) {
    const bool is_norm = i == nv;
    const cx<T>* Vi = V + (size_t)(is_norm ? 0 : i) * n;
    T ar = T(0), ai = T(0);
    size_t e = s0 + lane;
    for (; e + 96 < s1; e += 128) {
      cx<T> wv[4], vv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) wv[k] = ldcg(w + e + 32 * k);
      if (!is_norm) {
#pragma unroll
        for (int k = 0; k < 4; ++k) vv[k] = ldcg(Vi + e + 32 * k);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) vv[k] = wv[k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ar += vv[k].re * wv[k].re + vv[k].im * wv[k].im;
        ai += vv[k].re * wv[k].im - vv[k].im * wv[k].re;
      }
    }
    for (; e < s1; e += 32) {
      const cx<T> wv = ldcg(w + e);
      const cx<T> vv = is_norm ? wv : ldcg(Vi + e);
      ar += vv.re * wv.re + vv.im * wv.im;
      ai += vv.re * wv.im - vv.im * wv.re;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) {
      if (is_norm) {
        part[(size_t)(2 * nv) * G + bid] = double(ar);
      } else {
        part[(size_t)(2 * i) * G + bid] = double(ar);
        part[(size_t)(2 * i + 1) * G + bid] = double(ai);
      }
    }
  }
}

constexpr size_t kLargeSlice = 8 * NT;  // slices above this use the element-parallel update
constexpr size_t kStreamSlice = 2 * NT; // slices above this use the streaming dots (measured on GB300:
                                        // warp-split dots win for slices of a few hundred elements)

// Streaming variant for large slices: the slice is taken in blocks of EPT * NT elements; every
// thread keeps its EPT values of w in registers and streams the basis one vector at a time
// (EPT loads in flight per vector), accumulating 16 vectors per chunk before one warp
// transpose-reduction and a fixed-order block combine per chunk.
// FP32 streaming dots with the basis arriving through the cp.async ring (kStages - 1 vector blocks
// in flight per thread instead of one); otherwise the same sums in the same order as dots_stream.
__device__ void dots_stream_async(const cx<float>* V, size_t n, int nv, const cx<float>* w, double* part,
                                  bool with_norm, double* wred, unsigned bid, unsigned G, cx<float>* ring) {
  constexpr int EPT = 8, CH = 16;
  constexpr size_t BLK = (size_t)EPT * NT;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  size_t s0, s1;
  my_slice(n, bid, G, s0, s1);
  const int nblk = (int)((s1 - s0 + BLK - 1) / BLK);
  const int chunks = nv > 0 ? (nv + CH - 1) / CH : (with_norm ? 1 : 0);
  for (int c = 0; c < chunks; ++c) {
    const int c0 = c * CH;
    const int cnt = max(0, min(CH, nv - c0));
    const bool nrm = with_norm && c == 0;
    const int total = nblk * cnt;  // stream positions t = block * cnt + vector
    auto issue = [&](int t) {
      if (t < total) {
        const int bi = t / cnt, i = t - bi * cnt;
        const size_t blk = s0 + (size_t)bi * BLK;
        const cx<float>* Vi = V + (size_t)(c0 + i) * n;
        cx<float>* stg = ring + (size_t)(t % kStages) * BLK;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const size_t e = blk + threadIdx.x + (size_t)k * NT;
          if (e < s1) cp_async8(stg + threadIdx.x + k * NT, Vi + e);
        }
      }
      cp_async_commit();
    };
    for (int t = 0; t < kStages - 1; ++t) issue(t);
    float acc[2 * CH];
#pragma unroll
    for (int q = 0; q < 2 * CH; ++q) acc[q] = 0.f;
    float wn = 0.f;
    for (int bi = 0; bi < nblk; ++bi) {
      const size_t blk = s0 + (size_t)bi * BLK;
      cx<float> wv[EPT];
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const size_t e = blk + threadIdx.x + (size_t)k * NT;
        wv[k] = e < s1 ? ldcg(w + e) : mk<float>(0.f, 0.f);
        if (nrm) wn += wv[k].re * wv[k].re + wv[k].im * wv[k].im;
      }
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        if (i < cnt) {
          const int t = bi * cnt + i;
          issue(t + kStages - 1);
          cp_async_wait<kStages - 1>();
          const cx<float>* stg = ring + (size_t)(t % kStages) * BLK;
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const size_t e = blk + threadIdx.x + (size_t)k * NT;
            const cx<float> v = e < s1 ? stg[threadIdx.x + k * NT] : mk<float>(0.f, 0.f);
            acc[2 * i] += v.re * wv[k].re + v.im * wv[k].im;
            acc[2 * i + 1] += v.re * wv[k].im - v.im * wv[k].re;
          }
        }
      }
    }
    cp_async_wait<0>();
    const float ws = warp_tsum<float, 2 * CH>(acc);
    wred[wid * 2 * CH + lane] = double(ws);
    if (nrm) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wn += __shfl_xor_sync(0xffffffffu, wn, o);
      if (lane == 0) wred[NW * 2 * CH + wid] = double(wn);
    }
    __syncthreads();
    if (threadIdx.x < 2 * CH && (threadIdx.x >> 1) < cnt) {
      double t = 0;
      for (int q = 0; q < NW; ++q) t += wred[q * 2 * CH + threadIdx.x];
      part[(size_t)(2 * c0 + threadIdx.x) * G + bid] = t;
    }
    if (nrm && threadIdx.x == 0) {
      double t = 0;
      for (int q = 0; q < NW; ++q) t += wred[NW * 2 * CH + q];
      part[(size_t)(2 * nv) * G + bid] = t;
    }
    __syncthreads();
  }
}

template <typename T>
__device__ void dots_stream(const cx<T>* V, size_t n, int nv, const cx<T>* w, double* part, int pstride,
                            bool with_norm, double* wred, unsigned bid, unsigned G) {
  constexpr int EPT = 8, CH = 16;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  size_t s0, s1;
  my_slice(n, bid, G, s0, s1);
  const int chunks = nv > 0 ? (nv + CH - 1) / CH : (with_norm ? 1 : 0);
  for (int c = 0; c < chunks; ++c) {
    const int c0 = c * CH;
    const int cnt = max(0, min(CH, nv - c0));
    const bool nrm = with_norm && c == 0;
    T acc[2 * CH];
#pragma unroll
    for (int q = 0; q < 2 * CH; ++q) acc[q] = T(0);
    T wn = T(0);
    for (size_t blk = s0; blk < s1; blk += (size_t)EPT * NT) {
      cx<T> wv[EPT];
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const size_t e = blk + threadIdx.x + (size_t)k * NT;
        wv[k] = e < s1 ? ldcg(w + e) : mk<T>(T(0), T(0));
        if (nrm) wn += wv[k].re * wv[k].re + wv[k].im * wv[k].im;
      }
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        if (i < cnt) {
          const cx<T>* Vi = V + (size_t)(c0 + i) * n;
          cx<T> v[EPT];
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const size_t e = blk + threadIdx.x + (size_t)k * NT;
            v[k] = e < s1 ? ldcg(Vi + e) : mk<T>(T(0), T(0));
          }
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            acc[2 * i] += v[k].re * wv[k].re + v[k].im * wv[k].im;
            acc[2 * i + 1] += v[k].re * wv[k].im - v[k].im * wv[k].re;
          }
        }
      }
    }
    const T ws = warp_tsum<T, 2 * CH>(acc);
    wred[wid * 2 * CH + lane] = double(ws);
    if (nrm) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wn += __shfl_xor_sync(0xffffffffu, wn, o);
      if (lane == 0) wred[NW * 2 * CH + wid] = double(wn);
    }
    __syncthreads();
    if (threadIdx.x < 2 * CH && (threadIdx.x >> 1) < cnt) {
      double t = 0;
      for (int q = 0; q < NW; ++q) t += wred[q * 2 * CH + threadIdx.x];
      part[(size_t)(2 * c0 + threadIdx.x) * G + bid] = t;
    }
    if (nrm && threadIdx.x == 0) {
      double t = 0;
      for (int q = 0; q < NW; ++q) t += wred[NW * 2 * CH + q];
      part[(size_t)(2 * nv) * G + bid] = t;
    }
    __syncthreads();
  }
}

template <typename T>
__device__ void dots_pass(const cx<T>* V, size_t n, int nv, const cx<T>* w, double* part, int pstride, bool with_norm,
                          double* wred, unsigned bid, unsigned G, void* ring = nullptr) {
  if ((n + G - 1) / G > kStreamSlice) {
    if constexpr (sizeof(T) == 4) {
      if (ring) {
        dots_stream_async(V, n, nv, w, part, with_norm, wred, bid, G, reinterpret_cast<cx<float>*>(ring));
        return;
      }
    }
    dots_stream<T>(V, n, nv, w, part, pstride, with_norm, wred, bid, G);
  } else {
    dots_warp<T>(V, n, nv, w, part, pstride, with_norm, bid, G);
  }
}

// x[e] (+/-)= sum_i c_i V_i[e]; 8 vectors per step with all loads issued first (8 in flight).
// The vectors are visited from V_{nv-1} down to V_0: the Gram-Schmidt dots just read the basis
// upwards, so the most recently read vectors (still in L2) come first.
template <typename T, bool SUB>
__device__ __forceinline__ cx<T> axpy_all(cx<T> x, const cx<T>* V, size_t n, int nv, const T* sc, size_t e) {
  int r = 0;
  for (; r + 7 < nv; r += 8) {
    cx<T> v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = ldcg(V + (size_t)(nv - 1 - r - u) * n + e);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = nv - 1 - r - u;
      const T cr = sc[2 * i], ci = sc[2 * i + 1];
      const T pr = cr * v[u].re - ci * v[u].im, pi = cr * v[u].im + ci * v[u].re;
      if (SUB) {
        x.re -= pr;
        x.im -= pi;
      } else {
        x.re += pr;
        x.im += pi;
      }
    }
  }
  for (; r < nv; ++r) {
    const int i = nv - 1 - r;
    const cx<T> v = ldcg(V + (size_t)i * n + e);
    const T cr = sc[2 * i], ci = sc[2 * i + 1];
    const T pr = cr * v.re - ci * v.im, pi = cr * v.im + ci * v.re;
    if (SUB) {
      x.re -= pr;
      x.im -= pi;
    } else {
      x.re += pr;
      x.im += pi;
    }
  }
  return x;
}

// w -= sum_i h_i V_i over this CTA's slice with coefficients sc (typed), by threads
// t0 = 0 .. nthr - 1 of the CTA (no CTA-wide synchronisation inside, so a subset of the warps can
// run it while others do something else).
template <typename T>
__device__ __forceinline__ void update_slice(const cx<T>* V, size_t n, int nv, const T* sc, cx<T>* w, unsigned bid,
                                             unsigned G, int t0, int nthr) {
  size_t s0, s1;
  my_slice(n, bid, G, s0, s1);
  if (s1 - s0 > kLargeSlice) {
    // 8 elements per thread, two basis vectors per step (16 loads in flight), downwards: the
    // last-read vectors are still in L2; each element's updates keep the order V_{nv-1} .. V_0
    constexpr int E = 8;
    for (size_t e0 = s0 + t0; e0 < s1; e0 += (size_t)E * nthr) {
      cx<T> x[E];
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const size_t e = e0 + (size_t)k * nthr;
        x[k] = e < s1 ? ldcg(w + e) : mk<T>(T(0), T(0));
      }
      int i = nv - 1;
      for (; i >= 1; i -= 2) {
        const cx<T>* Va = V + (size_t)i * n;
        const cx<T>* Vb = V + (size_t)(i - 1) * n;
        cx<T> va[E], vb[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const size_t e = e0 + (size_t)k * nthr;
          va[k] = e < s1 ? ldcg(Va + e) : mk<T>(T(0), T(0));
          vb[k] = e < s1 ? ldcg(Vb + e) : mk<T>(T(0), T(0));
        }
        const T ar = sc[2 * i], ai = sc[2 * i + 1], br = sc[2 * i - 2], bi = sc[2 * i - 1];
#pragma unroll
        for (int k = 0; k < E; ++k) {
          x[k].re -= ar * va[k].re - ai * va[k].im;
          x[k].im -= ar * va[k].im + ai * va[k].re;
          x[k].re -= br * vb[k].re - bi * vb[k].im;
          x[k].im -= br * vb[k].im + bi * vb[k].re;
        }
      }
      if (i == 0) {
        const T cr = sc[0], ci = sc[1];
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const size_t e = e0 + (size_t)k * nthr;
          const cx<T> v = e < s1 ? ldcg(V + e) : mk<T>(T(0), T(0));
          x[k].re -= cr * v.re - ci * v.im;
          x[k].im -= cr * v.im + ci * v.re;
        }
      }
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const size_t e = e0 + (size_t)k * nthr;
        if (e < s1) w[e] = x[k];
      }
    }
  } else {
    for (size_t e = s0 + t0; e < s1; e += nthr) w[e] = axpy_all<T, true>(ldcg(w + e), V, n, nv, sc, e);
  }
}

// w -= sum_i h_i V_i over this CTA's slice (h in FP64 shared memory), all threads
template <typename T>
__device__ void update_pass(const cx<T>* V, size_t n, int nv, const double* h, T* sc, cx<T>* w, unsigned bid,
                            unsigned G) {
  for (int i = threadIdx.x; i < 2 * nv; i += NT) sc[i] = T(h[i]);
  __syncthreads();
  update_slice<T>(V, n, nv, sc, w, bid, G, threadIdx.x, NT);
}

// One Givens step on Hessenberg column j (entries h[0..2j+1] plus, with h2, a second-pass
// correction), subdiagonal hn2 = |h_{j+1,j}|^2, in the arithmetic type G_ with the rotation
// state (gc, gs, g) held in shared memory in that type.  Leaves the rotated column in col
// (FP64, CTA 0 only), the residual estimate |g_{j+1}|, the stop flag and 1/h_{j+1,j}.
template <typename G_>
__device__ void givens_step(int j, int cap, const G_* h, const G_* h2, double hn2, G_* col, G_* gc, G_* gs, G_* g,
                            double tol_abs, double* est, int* stop, double* scale) {
  // rotations i < j applied to the new column: the second entry of rotation i is the first
  // entry of rotation i + 1, so it travels in registers.  The other operands of 4 rotations are
  // loaded into registers before the 4 steps run (the column stores could otherwise alias the
  // next loads and serialise every step on shared-memory latency).
  // hn and the scale in the arithmetic type (FP64 square roots and divisions are slow here)
  const G_ hn = hn2 > 0 ? sqrt(G_(hn2)) : G_(0);
  G_ ar = h[0] + (h2 ? h2[0] : G_(0)), ai = h[1] + (h2 ? h2[1] : G_(0));
  constexpr int GB = 4;
  for (int i0 = 0; i0 < j; i0 += GB) {
    G_ bR[GB], bI[GB], cC[GB], sR[GB], sI[GB];
#pragma unroll
    for (int u = 0; u < GB; ++u) {
      const int i = min(i0 + u, j - 1);  // in-range index; steps past j - 1 are skipped below
      bR[u] = h[2 * i + 2] + (h2 ? h2[2 * i + 2] : G_(0));
      bI[u] = h[2 * i + 3] + (h2 ? h2[2 * i + 3] : G_(0));
      cC[u] = gc[i];
      sR[u] = gs[2 * i];
      sI[u] = gs[2 * i + 1];
    }
#pragma unroll
    for (int u = 0; u < GB; ++u) {
      if (i0 + u < j) {
        const G_ br = bR[u], bi = bI[u], c = cC[u], sr = sR[u], si = sI[u];
        // (a, b) <- (c a + s b, -conj(s) a + c b)
        col[2 * (i0 + u)] = c * ar + (sr * br - si * bi);
        col[2 * (i0 + u) + 1] = c * ai + (sr * bi + si * br);
        const G_ nr = -(sr * ar + si * ai) + c * br;
        const G_ ni = -(sr * ai - si * ar) + c * bi;
        ar = nr;
        ai = ni;
      }
    }
  }
  const G_ aa = sqrt(ar * ar + ai * ai);
  const G_ tt = sqrt(aa * aa + hn * hn);
  G_ c, sr, si;
  if (tt == G_(0)) {
    c = G_(1);
    sr = si = G_(0);
  } else if (aa == G_(0)) {
    c = G_(0);
    sr = G_(1);
    si = G_(0);
  } else {
    c = aa / tt;
    sr = (ar / aa) * hn / tt;
    si = (ai / aa) * hn / tt;
  }
  gc[j] = c;
  gs[2 * j] = sr;
  gs[2 * j + 1] = si;
  col[2 * j] = c * ar + sr * hn;
  col[2 * j + 1] = c * ai + si * hn;
  const G_ gr = g[2 * j], gi = g[2 * j + 1];
  const G_ g2r = -(sr * gr + si * gi), g2i = -(sr * gi - si * gr);
  g[2 * j + 2] = g2r;
  g[2 * j + 3] = g2i;
  g[2 * j] = c * gr;
  g[2 * j + 1] = c * gi;
  const double e = double(sqrt(g2r * g2r + g2i * g2i));
  *est = e;
  *stop = (e <= tol_abs || hn == G_(0) || j + 1 == cap || !(e == e)) ? 1 : 0;
  *scale = hn > G_(0) ? double(G_(1) / hn) : 0.0;
}

// The same Givens step run by all 32 lanes of warp 0.  The rotations i < j act on the new column
// as a linear recurrence of the carried entry, x_{i+1} = -conj(s_i) x_i + c_i h_{i+1} (the rotated
// entry i is c_i x_i + s_i h_{i+1}): each lane composes the affine maps of a block of consecutive
// rotations, a shuffle scan over the lanes gives every block its incoming x, and each lane then
// rotates its own block.  Lane 0 forms the new rotation.  Same outputs as givens_step.
template <typename G_>
__device__ void givens_step_warp(int j, int cap, const G_* h, const G_* h2, double hn2, G_* col, G_* gc, G_* gs,
                                 G_* g, double tol_abs, double* est, int* stop, double* scale) {
  const int lane = threadIdx.x & 31;
  const G_ hn = hn2 > 0 ? sqrt(G_(hn2)) : G_(0);
  const int B = (j + 31) / 32;
  const int i0 = min(lane * B, j), i1 = min(i0 + B, j);
  const G_ x0r = h[0] + (h2 ? h2[0] : G_(0)), x0i = h[1] + (h2 ? h2[1] : G_(0));
  // composite map x -> A x + Bv of this lane's block
  G_ Ar = G_(1), Ai = G_(0), Br = G_(0), Bi = G_(0);
  for (int i = i0; i < i1; ++i) {
    const G_ c = gc[i], sr = gs[2 * i], si = gs[2 * i + 1];
    const G_ br = h[2 * i + 2] + (h2 ? h2[2 * i + 2] : G_(0)), bi = h[2 * i + 3] + (h2 ? h2[2 * i + 3] : G_(0));
    const G_ pr = -sr, pi = si;  // -conj(s)
    const G_ nAr = pr * Ar - pi * Ai, nAi = pr * Ai + pi * Ar;
    const G_ nBr = (pr * Br - pi * Bi) + c * br, nBi = (pr * Bi + pi * Br) + c * bi;
    Ar = nAr;
    Ai = nAi;
    Br = nBr;
    Bi = nBi;
  }
  // inclusive scan: lane l holds the map of blocks 0..l
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const G_ qAr = __shfl_up_sync(0xffffffffu, Ar, off), qAi = __shfl_up_sync(0xffffffffu, Ai, off);
    const G_ qBr = __shfl_up_sync(0xffffffffu, Br, off), qBi = __shfl_up_sync(0xffffffffu, Bi, off);
    if (lane >= off) {  // mine after theirs: x -> A (qA x + qB) + B
      const G_ nBr = (Ar * qBr - Ai * qBi) + Br, nBi = (Ar * qBi + Ai * qBr) + Bi;
      const G_ nAr = Ar * qAr - Ai * qAi, nAi = Ar * qAi + Ai * qAr;
      Ar = nAr;
      Ai = nAi;
      Br = nBr;
      Bi = nBi;
    }
  }
  // x entering this lane's block: the map of blocks 0..l-1 applied to x_0
  const G_ eAr = __shfl_up_sync(0xffffffffu, Ar, 1), eAi = __shfl_up_sync(0xffffffffu, Ai, 1);
  const G_ eBr = __shfl_up_sync(0xffffffffu, Br, 1), eBi = __shfl_up_sync(0xffffffffu, Bi, 1);
  G_ ar = x0r, ai = x0i;
  if (lane > 0) {
    ar = (eAr * x0r - eAi * x0i) + eBr;
    ai = (eAr * x0i + eAi * x0r) + eBi;
  }
  for (int i = i0; i < i1; ++i) {
    const G_ c = gc[i], sr = gs[2 * i], si = gs[2 * i + 1];
    const G_ br = h[2 * i + 2] + (h2 ? h2[2 * i + 2] : G_(0)), bi = h[2 * i + 3] + (h2 ? h2[2 * i + 3] : G_(0));
    col[2 * i] = c * ar + (sr * br - si * bi);
    col[2 * i + 1] = c * ai + (sr * bi + si * br);
    const G_ nr = -(sr * ar + si * ai) + c * br;
    const G_ ni = -(sr * ai - si * ar) + c * bi;
    ar = nr;
    ai = ni;
  }
  // x_j from the lane that rotated index j - 1 (lane 0 when j == 0)
  const int last = j > 0 ? (j - 1) / B : 0;
  ar = __shfl_sync(0xffffffffu, ar, last);
  ai = __shfl_sync(0xffffffffu, ai, last);
  if (lane != 0) return;
  const G_ aa = sqrt(ar * ar + ai * ai);
  const G_ tt = sqrt(aa * aa + hn * hn);
  G_ c, sr, si;
  if (tt == G_(0)) {
    c = G_(1);
    sr = si = G_(0);
  } else if (aa == G_(0)) {
    c = G_(0);
    sr = G_(1);
    si = G_(0);
  } else {
    c = aa / tt;
    sr = (ar / aa) * hn / tt;
    si = (ai / aa) * hn / tt;
  }
  gc[j] = c;
  gs[2 * j] = sr;
  gs[2 * j + 1] = si;
  col[2 * j] = c * ar + sr * hn;
  col[2 * j + 1] = c * ai + si * hn;
  const G_ gr = g[2 * j], gi = g[2 * j + 1];
  const G_ g2r = -(sr * gr + si * gi), g2i = -(sr * gi - si * gr);
  g[2 * j + 2] = g2r;
  g[2 * j + 3] = g2i;
  g[2 * j] = c * gr;
  g[2 * j + 1] = c * gi;
  const double e = double(sqrt(g2r * g2r + g2i * g2i));
  *est = e;
  *stop = (e <= tol_abs || hn == G_(0) || j + 1 == cap || !(e == e)) ? 1 : 0;
  *scale = hn > G_(0) ? double(G_(1) / hn) : 0.0;
}

template <typename T, int R, bool CL, int TS = 0>
__global__ void __launch_bounds__(NT) k_gmres(OpP<T> P, const cx<T>* __restrict__ b, cx<T>* __restrict__ x,
                                              cx<T>* V, cx<T>* w0, cx<T>* w1, double* partA, double* partB,
                                              int pstride, double* Rg, hz::GmresState* st, int cap, double tol,
                                              double eta2) {
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t n = (size_t)P.nx * P.ny;
  // CTAs that share this solve: the cluster (one right-hand side per cluster) or the whole grid
  unsigned bid, G;
  if constexpr (CL) {
    unsigned q;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(bid));
    asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(G));
    asm("mov.u32 %0, %%clusterid.x;" : "=r"(q));
    const size_t rgs = 2 * (size_t)cap * (cap + 1) + 2 * (size_t)cap + 3 * (size_t)pstride;
    b += q * n;
    x += q * n;
    V += q * (size_t)(cap + 1) * n;
    w0 += q * n;
    w1 += q * n;
    partA += (size_t)q * G * pstride;
    partB += (size_t)q * G * pstride;
    Rg += q * rgs;
    st += q;
    P.k += q * P.kstride;
  } else {
    bid = blockIdx.x;
    G = gridDim.x;
  }
  timing_begin(st, bid);
  constexpr int TOX = TileShape<TS>::X, TOY = TileShape<TS>::Y;
  const int tilesx = (P.nx + TOX - 1) / TOX, tilesy = (P.ny + TOY - 1) / TOY;
  const int ntiles = tilesx * tilesy;
  // the operator tile, and for FP32 the cp.async ring of the vector phases, share the first region
  constexpr size_t kTileRegion = tile_smem_bytes<T, R>(TOX, TOY);
  constexpr size_t kRegion = (sizeof(T) == 4 && kRingBytes > kTileRegion) ? kRingBytes : kTileRegion;
  void* ring = sizeof(T) == 4 ? (void*)smem : nullptr;
  unsigned char* kp = smem + kRegion;
  KShared K;
  K.h = reinterpret_cast<double*>(kp);
  K.h1 = K.h + 2 * (cap + 1) + 2;
  K.gc = K.h1 + 2 * (cap + 1) + 2;  // (FP64 slots reused as typed Givens state below)
  K.gs = K.gc + cap;
  K.g = K.gs + 2 * cap;
  K.wred = K.g + 2 * (cap + 1);
  K.scal = K.wred + kWred;
  K.flags = reinterpret_cast<int*>(K.scal + 4);
  T* sc = reinterpret_cast<T*>(K.flags + 4);
  T* gcT = reinterpret_cast<T*>(K.gc);      // cap cosines
  T* gsT = reinterpret_cast<T*>(K.gs);      // 2 cap sines
  T* gT = reinterpret_cast<T*>(K.g);        // 2 (cap + 1) rotated right-hand side
  T* colT = sc + 2 * (cap + 1);             // 2 (cap + 1) rotated column
  T* hT = colT + 2 * (cap + 1);             // 2 (cap + 1) + 2 coefficients in the arithmetic type
  T* h1T = hT + 2 * (cap + 1) + 2;          // 2 (cap + 1) first-pass coefficients
  double* red = Rg + 2 * (size_t)cap * (cap + 1) + 2 * (size_t)cap;  // 3 * pstride reduced values

  // beta = ||b||
  dots_pass<T>(V, n, 0, b, partA, pstride, true, K.wred, bid, G);
  if (!reduce_all<CL>(st, G, partA, pstride, 1, red, K.scal + 1)) return;
  const double beta = sqrt(K.scal[1]);
  if (!(beta > 0)) {
    if (bid == 0 && threadIdx.x == 0) {
      st->its = 0;
      st->est = 0;
    }
    return;
  }
  const double tol_abs = tol * beta;
  if (threadIdx.x == 0) {
    gT[0] = T(beta);
    gT[1] = T(0);
  }
  const cx<T>* src = b;
  double s = 1.0 / beta;
  cx<T>* wcur = w0;
  cx<T>* wnext = w1;
  int jstop = 0;
  double est = beta;
  // algorithmic bytes of this solve in units of one vector (e n): ||b|| reads b once
  const double eb = (double)sizeof(cx<T>), ekb = (double)sizeof(T);
  double vec_units = 1.0, k_units = 0.0;
  int reorths = 0;
  for (int j = 0; j < cap; ++j) {
    // op: V_j = s * src (own tile nodes), wnext = M_l V_j
    cx<T>* Vj = V + (size_t)j * n;
    TilePrefetch<T, R, TOX, TOY> pf;
    if ((int)bid < ntiles) pf.load(P, src, ((int)bid % tilesx) * TOX, ((int)bid / tilesx) * TOY);
    for (int t = bid; t < ntiles; t += G) {
      const int ox0 = (t % tilesx) * TOX, oy0 = (t / tilesx) * TOY;
      TileView<T, R> tv = make_tile<T, R>(smem, TOX, TOY, ox0, oy0);
      pf.store(tv, T(s));
      __syncthreads();
      if (t + (int)G < ntiles) pf.load(P, src, ((t + G) % tilesx) * TOX, ((t + G) / tilesx) * TOY);
      tile_finish<T, R>(tv, P);
      if (R == 1) {
        for (int q = threadIdx.x; q < TOX * TOY; q += NT) {
          const int ox = q % TOX, oy = q / TOX;
          const int gx = ox0 + ox, gy = oy0 + oy;
          if (gx >= P.nx || gy >= P.ny) continue;
          const size_t i = (size_t)gy * P.nx + gx;
          wnext[i] = tile_op<T, R>(tv, P, ox, oy);
          Vj[i] = tv.u(ox + R, oy + R);
        }
      } else {
        for (int q = threadIdx.x; q < TOX * (TOY / 4); q += NT) {
          const int ox = q % TOX, sy = (q / TOX) * 4;
          const int cnt = min(4, P.ny - (oy0 + sy));
          if (ox0 + ox >= P.nx || cnt <= 0) continue;
          cx<T> v[4];
          tile_op_seg<T, R>(tv, P, ox, sy, cnt, v);
          for (int k = 0; k < cnt; ++k) {
            const size_t i = (size_t)(oy0 + sy + k) * P.nx + (ox0 + ox);
            wnext[i] = v[k];
            Vj[i] = tv.u(ox + R, sy + k + R);
          }
        }
      }
      __syncthreads();
    }
    if (!bar_all<CL>(st, G)) return;
    vec_units += 3.0;  // read src, write V_j and w
    k_units += 1.0;
    // h = V^H w and ||w||^2; ||w'||^2 = ||w||^2 - sum |h_i|^2 (Pythagoras) unless the vector
    // loses more than reorth_eta of its norm, in which case a second classical pass runs
    const int nv = j + 1;
    vec_units += nv + 1;  // read V_0..V_j and w
    dots_pass<T>(V, n, nv, wnext, partA, pstride, true, K.wred, bid, G, ring);
    if (!reduce_all<CL>(st, G, partA, pstride, 2 * nv + 1, red, K.h)) return;
    bool updated = false;
    {
      // every thread holds the same reduced values, so every thread takes the same decision
      const T hs = typed_copy_sumsq<T>(K.h, hT, 2 * nv, 2 * nv, hT + 2 * (cap + 1) + 1);
      const double wn2 = K.h[2 * nv];
      const double hp = wn2 - double(hs);
      if (hp >= eta2 * wn2) {
        // one pass suffices: warp 0 runs the Givens step while the other warps already apply
        // w' = w - V h (not needed if the solve stops here; it is then simply unused)
        for (int i = threadIdx.x; i < 2 * nv; i += NT) sc[i] = T(K.h[i]);
        __syncthreads();
        if (threadIdx.x < 32) {
          if (threadIdx.x == 0) {
            K.scal[3] = hp;
            K.flags[1] = 0;
          }
          givens_step_warp<T>(j, cap, hT, (const T*)nullptr, hp, colT, gcT, gsT, gT, tol_abs, K.scal + 2, K.flags,
                              K.scal);
        } else {
          update_slice<T>(V, n, nv, sc, wnext, bid, G, threadIdx.x - 32, NT - 32);
        }
        updated = true;
      } else if (threadIdx.x == 0) {
        K.scal[3] = hp;
        K.flags[1] = 1;
      }
    }
    __syncthreads();
    if (K.flags[1]) {  // second classical pass
      ++reorths;
      vec_units += (nv + 2) + (nv + 1);  // w -= V h (read V, w; write w), then V^H w again
      update_pass<T>(V, n, nv, K.h, sc, wnext, bid, G);
      if (!bar_all<CL>(st, G)) return;
      for (int i = threadIdx.x; i < 2 * nv; i += NT) h1T[i] = hT[i];
      dots_pass<T>(V, n, nv, wnext, partA, pstride, true, K.wred, bid, G, ring);
      if (!reduce_all<CL>(st, G, partA, pstride, 2 * nv + 1, red, K.h)) return;
      const T hs = typed_copy_sumsq<T>(K.h, hT, 2 * nv, 2 * nv, hT + 2 * (cap + 1) + 1);
      if (threadIdx.x < 32) {
        const double hp = K.h[2 * nv] - double(hs);
        givens_step_warp<T>(j, cap, h1T, hT, hp, colT, gcT, gsT, gT, tol_abs, K.scal + 2, K.flags, K.scal);
      }
      __syncthreads();
    }
    if (bid == 0) {  // CTA 0 keeps the rotated column j (FP64) for the final triangular solve
      double* Rc = Rg + 2 * (size_t)j * (cap + 1);
      for (int i = threadIdx.x; i < 2 * nv; i += NT) Rc[i] = double(colT[i]);
    }
    if (!K.flags[0]) {  // w' = w - V h (with the last pass's coefficients); the next op needs it complete
      vec_units += nv + 2;
      if (!updated) update_pass<T>(V, n, nv, K.h, sc, wnext, bid, G);
      if (!bar_all<CL>(st, G)) return;
    }
    est = K.scal[2];
    if (K.flags[0]) {
      jstop = j + 1;
      break;
    }
    s = K.scal[0];
    src = wnext;
    cx<T>* tmp = wcur;
    wcur = wnext;
    wnext = tmp;
  }
  // y = R^-1 g by warp 0 of CTA 0 (column-oriented back substitution: lane 0 divides, the
  // warp updates the remaining right-hand side from column i of R), then x += V y everywhere.
  // Every thread of CTA 0 wrote part of the last column of R just before the loop ended (a
  // stopping iteration takes no barrier), so the CTA synchronises before warp 0 reads it.
  __syncthreads();
  double* y = Rg + 2 * (size_t)cap * (cap + 1);
  if (bid == 0 && threadIdx.x < 32) {  // Rg was written by this CTA; y is read after the barrier
    const int lane = threadIdx.x;
    double* gw = K.h;     // working right-hand side, FP64
    double* dinv = K.h1;  // conj(R_ii) / |R_ii|^2, computed in parallel before the serial chain
    for (int i = lane; i < 2 * jstop; i += 32) gw[i] = double(gT[i]);
    for (int i = lane; i < jstop; i += 32) {
      const double dr = Rg[2 * ((size_t)i * (cap + 1) + i)], di = Rg[2 * ((size_t)i * (cap + 1) + i) + 1];
      const double d = dr * dr + di * di;
      dinv[2 * i] = dr / d;
      dinv[2 * i + 1] = -di / d;
    }
    __syncwarp();
    for (int i = jstop - 1; i >= 0; --i) {
      const double* Ri = Rg + 2 * (size_t)i * (cap + 1);  // R_{k,i}, k <= i
      double yr = 0, yi = 0;
      if (lane == 0) {
        const double sr = gw[2 * i], si = gw[2 * i + 1];
        const double ir = dinv[2 * i], ii = dinv[2 * i + 1];
        yr = sr * ir - si * ii;
        yi = sr * ii + si * ir;
        y[2 * i] = yr;
        y[2 * i + 1] = yi;
      }
      yr = __shfl_sync(0xffffffffu, yr, 0);
      yi = __shfl_sync(0xffffffffu, yi, 0);
      for (int k = lane; k < i; k += 32) {
        const double rr = Ri[2 * k], ri = Ri[2 * k + 1];
        gw[2 * k] -= rr * yr - ri * yi;
        gw[2 * k + 1] -= rr * yi + ri * yr;
      }
      __syncwarp();
    }
  }
  if (bid == 0 && threadIdx.x == 0) {
    st->its = jstop;
    st->est = est;
    st->total_its += jstop;
    st->total_reorth += reorths;
    // x += V y reads jstop basis vectors and x and writes x
    st->total_bytes += (vec_units + jstop + 2) * eb * (double)n + k_units * ekb * (double)n;
  }
  if (!bar_all<CL>(st, G)) return;
  for (int i = threadIdx.x; i < 2 * jstop; i += NT) sc[i] = T(__ldcg(y + i));
  __syncthreads();
  size_t s0, s1;
  my_slice(n, bid, G, s0, s1);
  for (size_t e = s0 + threadIdx.x; e < s1; e += NT) x[e] = axpy_all<T, false>(x[e], V, n, jstop, sc, e);
  timing_end(st, G);
}


// ---------------------------------------------------------------------------------------------
// Tile-owned form (levels whose tiling fits the grid): CTA b owns tile b of a tiling in which
// the last tile column / row absorbs the remainder (2^k + 1 grids split evenly).  The CTA
// keeps M_l V_j of its own nodes in shared memory, so the Gram-Schmidt dots, a second pass and
// the update touch only its own nodes: one grid barrier for the reduction and one after the
// update (halo exchange through the vector in global memory) per iteration.

__host__ __device__ inline int tiles_along(int n, int t) { return n > 1 ? (n - 1 + t - 1) / t : 1; }

struct TileGrid {
  int TX, TY, ntx, nty;
};

template <typename T>
struct ScaledSrc {
  const cx<T>* x;
  int nx;
  T s;
  __device__ __forceinline__ cx<T> operator()(int gx, int gy) const { return s * ldcg(x + (size_t)gy * nx + gx); }
};

struct OwnNodes {  // own node q (row-major in the tile) -> grid index
  int OX, OY, ox0, oy0, nx;
  __device__ __forceinline__ size_t operator()(int q) const {
    const int oy = q / OX, ox = q - oy * OX;
    return (size_t)(oy0 + oy) * nx + (ox0 + ox);
  }
  __device__ __forceinline__ int count() const { return OX * OY; }
};

// ---------------------------------------------------------------------------------------------
// Tile-owned form with one grid barrier per iteration.  CTA b owns tile b of a tiling in which the
// last tile column / row absorbs the remainder (2^k + 1 grids split evenly).  Per iteration:
//   op      V_j = s w at the own nodes (w kept in shared memory) and the halo (read from the
//           neighbours' w in global memory once their flags say it is complete), z = M_l V_j
//           kept in shared memory;
//   dots    h = V^H z and ||z||^2 over the own nodes;
//   reduce  the grid barrier: every CTA sums all CTA partials itself in one fixed order;
//   update  w = z - V h at the own nodes, written to global memory for the neighbours' halos,
//           then the CTA raises its flag to j + 1 (warp 0 meanwhile runs the serial Givens step).
// The halo exchange waits only for the (at most eight) neighbouring tiles, not for the whole
// grid.  The first nres basis vectors of the own nodes stay in shared memory (all of them where
// they fit), so the dots, the updates and the final x += V y read those from shared memory;
// vectors beyond nres live in global memory.  Partial sums alternate between two buffers by a
// running count of reductions, so a buffer is rewritten only after every CTA passed the barrier
// that follows its last read.

// x - sum_{i < nv} c_i V_i, the basis visited from V_{nv-1} down to V_0, 8 loads in flight; ld(i)
// returns V_i at the node.
template <typename T, class LD>
__device__ __forceinline__ cx<T> sub_comb(cx<T> x, int nv, const T* sc, const LD& ld) {
  int r = 0;
  for (; r + 7 < nv; r += 8) {
    cx<T> v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = ld(nv - 1 - r - u);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = nv - 1 - r - u;
      const T cr = sc[2 * i], ci = sc[2 * i + 1];
      x.re -= cr * v[u].re - ci * v[u].im;
      x.im -= cr * v[u].im + ci * v[u].re;
    }
  }
  for (; r < nv; ++r) {
    const int i = nv - 1 - r;
    const cx<T> v = ld(i);
    const T cr = sc[2 * i], ci = sc[2 * i + 1];
    x.re -= cr * v.re - ci * v.im;
    x.im -= cr * v.im + ci * v.re;
  }
  return x;
}

template <typename T>
struct OwnBasis {  // V_i at own node q (grid node e): shared memory below nres, global above
  const cx<T>* Vs;
  const cx<T>* V;
  int stride, q, nres;
  size_t n, e;
  __device__ __forceinline__ cx<T> operator()(int i) const {
    return i < nres ? Vs[i * stride + q] : ldcg(V + (size_t)i * n + e);
  }
};

// Partials of h_i = V_i^H z (i < nv) and ||z||^2 over the own nodes (z in shared memory): warp w
// takes vectors w, w + NW, ... (the norm is job nv), its lanes stride over the own nodes, and a
// shuffle tree gives the CTA partial directly (no block-level combine), stored in the arithmetic
// type, value-major: part[i * G + b].
template <typename T>
__device__ void dots_own3(const cx<T>* V, const cx<T>* Vs, int vstride, int nres, size_t n, int nv,
                          const cx<T>* Wt, const OwnNodes& on, T* part, unsigned bid, unsigned G) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nown = on.count();
  for (int i = wid; i <= nv; i += NW) {
    T ar = T(0), ai = T(0);
    if (i == nv) {
      for (int q = lane; q < nown; q += 32) {
        const cx<T> z = Wt[q];
        ar += z.re * z.re + z.im * z.im;
      }
    } else if (i < nres) {
      const cx<T>* vi = Vs + (size_t)i * vstride;
      for (int q = lane; q < nown; q += 32) {
        const cx<T> v = vi[q], z = Wt[q];
        ar += v.re * z.re + v.im * z.im;
        ai += v.re * z.im - v.im * z.re;
      }
    } else {
      const cx<T>* vi = V + (size_t)i * n;
      for (int q = lane; q < nown; q += 32) {
        const cx<T> v = ldcg(vi + on(q)), z = Wt[q];
        ar += v.re * z.re + v.im * z.im;
        ai += v.re * z.im - v.im * z.re;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) {
      part[(size_t)(2 * i) * G + bid] = ar;
      if (i < nv) part[(size_t)(2 * i + 1) * G + bid] = ai;
    }
  }
}

// Grid barrier, then every CTA sums the typed partials part[i * G + b] over b itself for i < m,
// in one fixed order (4 lanes per value, 16-byte loads of 4 consecutive CTAs' partials when G is
// a multiple of 4), into out[] (FP64, shared); every CTA holds bitwise-identical sums.
template <typename T>
__device__ __forceinline__ bool grid_reduce_t(hz::GmresState* gs, unsigned G, const T* part, int m, double* out,
                                              T* outT = nullptr) {
  if (!grid_sync(gs, G)) return false;
  constexpr int K = 4;
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < m; base += NT / K) {
    const int i = base + (int)threadIdx.x / K;
    const int k = lane % K;
    T t = T(0);
    if (i < m) {
      const T* pi = part + (size_t)i * G;
      if constexpr (sizeof(T) == 4) {
        if ((G & 3u) == 0) {
          const float4* p4 = reinterpret_cast<const float4*>(pi);
          const int g4 = (int)G / 4;
          float4 a[8];
          int b = k;
          for (; b + 7 * K < g4; b += 8 * K) {
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = __ldcg(p4 + b + u * K);
#pragma unroll
            for (int u = 0; u < 8; ++u) t += (a[u].x + a[u].y) + (a[u].z + a[u].w);
          }
          for (; b < g4; b += K) {
            const float4 c = __ldcg(p4 + b);
            t += (c.x + c.y) + (c.z + c.w);
          }
        } else {
          for (int b = k; b < (int)G; b += K) t += __ldcg(pi + b);
        }
      } else {
        T a[8];
        int b = k;
        for (; b + 7 * K < (int)G; b += 8 * K) {
#pragma unroll
          for (int u = 0; u < 8; ++u) a[u] = __ldcg(pi + b + u * K);
#pragma unroll
          for (int u = 0; u < 8; ++u) t += a[u];
        }
        for (; b < (int)G; b += K) t += __ldcg(pi + b);
      }
    }
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (i < m && k == 0) {
      out[i] = double(t);
      if (outT) outT[i] = t;
    }
  }
  __syncthreads();
  return true;
}

// Sum of squares of v[0..m) by warp 0 into *sred, then a CTA barrier; returns it in every thread.
template <typename T>
__device__ __forceinline__ T warp0_sumsq(const T* v, int m, T* sred) {
  if (threadIdx.x < 32) {
    T acc = T(0);
    for (int i = threadIdx.x; i < m; i += 32) acc += v[i] * v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) *sred = acc;
  }
  __syncthreads();
  return *sred;
}

// Raise this CTA's halo flag to `val` after every thread's global writes (CTA barrier, then a
// GPU-scope fence by the signalling thread, as in the grid barrier).
__device__ __forceinline__ void flag_raise(unsigned* nflag, unsigned bid, unsigned val) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(nflag + bid, val);
  }
}

// Wait until the flags of the (at most eight) tiles around tile (tx, ty) reach `val`; one thread
// per neighbour, each spin bounded by the clock budget of the grid barrier.  Ends with a CTA
// barrier; false if a wait ran out (error flag set) or another CTA failed.
__device__ __forceinline__ bool wait_neighbours(hz::GmresState* gs, const unsigned* nflag, const TileGrid& tg, int tx,
                                                int ty, unsigned val) {
  if (threadIdx.x < 9 && threadIdx.x != 4) {
    const int nx_ = tx + (int)(threadIdx.x % 3) - 1, ny_ = ty + (int)(threadIdx.x / 3) - 1;
    if (nx_ >= 0 && nx_ < tg.ntx && ny_ >= 0 && ny_ < tg.nty) {
      const volatile unsigned* f = nflag + (ny_ * tg.ntx + nx_);
      const long long t0 = clock64();
      while (*f < val) {
        if (failed(gs)) break;
        if (clock64() - t0 > kSpinCycles) {
          atomicExch(&gs->err, 1);
          break;
        }
        __nanosleep(20);
      }
      __threadfence();
    }
  }
  __syncthreads();
  return !failed(gs);
}

template <typename T, int R>
__global__ void __launch_bounds__(NT) k_gmres_tile2(OpP<T> P, TileGrid tg, const cx<T>* __restrict__ b,
                                                    cx<T>* __restrict__ x, cx<T>* V, cx<T>* wbuf, unsigned* nflag,
                                                    double* partA, double* partB, double* Rg, hz::GmresState* st,
                                                    int cap, int nres, double tol, double eta2) {
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t n = (size_t)P.nx * P.ny;
  const unsigned bid = blockIdx.x, G = gridDim.x;
  timing_begin(st, bid);
  if (threadIdx.x == 0) nflag[bid] = 0u;  // ordered before every neighbour's wait by the first barrier
  const int tx = (int)bid % tg.ntx, ty = (int)bid / tg.ntx;
  OwnNodes on;
  on.ox0 = tx * tg.TX;
  on.oy0 = ty * tg.TY;
  on.OX = (tx == tg.ntx - 1) ? P.nx - on.ox0 : tg.TX;
  on.OY = (ty == tg.nty - 1) ? P.ny - on.oy0 : tg.TY;
  on.nx = P.nx;
  const int nown = on.count();
  const int vstride = (tg.TX + 1) * (tg.TY + 1);
  // shared memory: tile | own z / w | own basis V_0 .. V_{nres-1} | Krylov scratch
  cx<T>* Wt = reinterpret_cast<cx<T>*>(smem + tile_smem_bytes<T, R>(tg.TX + 1, tg.TY + 1));
  cx<T>* Vs = Wt + vstride;
  unsigned char* kp = reinterpret_cast<unsigned char*>(Vs + (size_t)nres * vstride);
  KShared K;
  K.h = reinterpret_cast<double*>(kp);
  K.h1 = K.h + 2 * (cap + 1) + 2;
  K.gc = K.h1 + 2 * (cap + 1) + 2;
  K.gs = K.gc + cap;
  K.g = K.gs + 2 * cap;
  K.wred = K.g + 2 * (cap + 1);
  K.scal = K.wred + kWred;
  K.flags = reinterpret_cast<int*>(K.scal + 4);
  T* sc = reinterpret_cast<T*>(K.flags + 4);
  T* gcT = reinterpret_cast<T*>(K.gc);
  T* gsT = reinterpret_cast<T*>(K.gs);
  T* gT = reinterpret_cast<T*>(K.g);
  T* colT = sc + 2 * (cap + 1);
  T* hT = colT + 2 * (cap + 1);
  T* h1T = hT + 2 * (cap + 1) + 2;
  const TileView<T, R> tv = make_tile<T, R>(smem, on.OX, on.OY, on.ox0, on.oy0);
  const int WX = on.OX + 2 * R, WY = on.OY + 2 * R;
  const int gx0 = on.ox0 - R, gy0 = on.oy0 - R;

  // beta = ||b|| over the own nodes, reduced over the grid; w_{-1} := b at the own nodes
  for (int q = threadIdx.x; q < nown; q += NT) Wt[q] = ldcg(b + on(q));
  __syncthreads();
  unsigned rc = 0;  // reductions so far: partial buffer rc & 1
  dots_own3<T>(V, Vs, vstride, 0, n, 0, Wt, on, reinterpret_cast<T*>(partA), bid, G);
  if (!grid_reduce_t<T>(st, G, reinterpret_cast<const T*>(partA), 1, K.scal + 1)) return;
  ++rc;
  const double beta = sqrt(K.scal[1]);
  if (!(beta > 0)) {
    if (bid == 0 && threadIdx.x == 0) {
      st->its = 0;
      st->est = 0;
    }
    return;
  }
  const double tol_abs = tol * beta;
  if (threadIdx.x == 0) {
    gT[0] = T(beta);
    gT[1] = T(0);
  }
  T s = T(1.0 / beta);
  const cx<T>* src = b;  // the vector the halo is read from: b, then the neighbours' w
  int jstop = 0;
  double est = beta;
  const double eb = (double)sizeof(cx<T>), ekb = (double)sizeof(T);
  double vec_units = 1.0, k_units = 0.0;
  int reorths = 0;
  for (int j = 0; j < cap; ++j) {
    // ---- op: V_j = s w (own cells from shared memory, halo cells from global memory), z = M V_j
    if (j > 0 && !wait_neighbours(st, nflag, tg, tx, ty, (unsigned)j)) return;
    for (int idx = threadIdx.x; idx < WX * WY; idx += NT) {
      const int cy = idx / WX, cxx = idx - cy * WX;
      const int ox = cxx - R, oy = cy - R;
      const int gx = gx0 + cxx, gy = gy0 + cy;
      cx<T> v = mk<T>(T(0), T(0));
      T kk = T(0);
      if (gx >= 0 && gx < P.nx && gy >= 0 && gy < P.ny) {
        const size_t e = (size_t)gy * P.nx + gx;
        const bool own = ox >= 0 && ox < on.OX && oy >= 0 && oy < on.OY;
        v = s * (own ? Wt[oy * on.OX + ox] : ldcg(src + e));
        if (R >= 2) kk = P.k[e];
      }
      tv.U[idx] = v;
      if (R >= 2) tv.W[idx] = (kk * kk) * v;
    }
    __syncthreads();
    tile_finish<T, R>(tv, P);
    cx<T>* Vj = V + (size_t)j * n;
    for (int it = threadIdx.x; it < on.OX * ((on.OY + 3) / 4); it += NT) {
      const int ox = it % on.OX, sy = (it / on.OX) * 4;
      const int cnt = min(4, on.OY - sy);
      cx<T> v[4];
      tile_op_seg<T, R>(tv, P, ox, sy, cnt, v);
      for (int k = 0; k < cnt; ++k) {
        const int q = (sy + k) * on.OX + ox;
        const cx<T> u = tv.u(ox + R, sy + k + R);
        Wt[q] = v[k];
        if (j < nres) Vs[j * vstride + q] = u;
        else Vj[on(q)] = u;
      }
    }
    __syncthreads();
    vec_units += 2.0;  // read the previous vector, write V_j (z stays on chip)
    k_units += 1.0;
    const int nv = j + 1;
    vec_units += nv;  // V_0..V_j
    T* part = reinterpret_cast<T*>((rc & 1) ? partB : partA);
    dots_own3<T>(V, Vs, vstride, nres, n, nv, Wt, on, part, bid, G);
    if (!grid_reduce_t<T>(st, G, part, 2 * nv + 1, K.h, hT)) return;
    ++rc;
    const double wn2 = K.h[2 * nv];
    double hp = wn2 - double(warp0_sumsq<T>(hT, 2 * nv, hT + 2 * (cap + 1) + 1));
    if (hp >= eta2 * wn2) {
      // one pass: warp 0 rotates while the other warps form w = z - V h at the own nodes
      if (threadIdx.x < 32) {
        givens_step_warp<T>(j, cap, hT, (const T*)nullptr, hp, colT, gcT, gsT, gT, tol_abs, K.scal + 2, K.flags,
                            K.scal);
      } else {
        for (int q = threadIdx.x - 32; q < nown; q += NT - 32) {
          const size_t e = on(q);
          const cx<T> w = sub_comb<T>(Wt[q], nv, hT, OwnBasis<T>{Vs, V, vstride, q, nres, n, e});
          Wt[q] = w;
          wbuf[e] = w;
        }
      }
      vec_units += nv + 1;
    } else {
      // second classical pass: w' = z - V h, h2 = V^H w', w'' = w' - V h2
      ++reorths;
      for (int i = threadIdx.x; i < 2 * nv; i += NT) h1T[i] = hT[i];
      for (int q = threadIdx.x; q < nown; q += NT)
        Wt[q] = sub_comb<T>(Wt[q], nv, hT, OwnBasis<T>{Vs, V, vstride, q, nres, n, on(q)});
      __syncthreads();
      T* part2 = reinterpret_cast<T*>((rc & 1) ? partB : partA);
      dots_own3<T>(V, Vs, vstride, nres, n, nv, Wt, on, part2, bid, G);
      if (!grid_reduce_t<T>(st, G, part2, 2 * nv + 1, K.h, hT)) return;
      ++rc;
      hp = K.h[2 * nv] - double(warp0_sumsq<T>(hT, 2 * nv, hT + 2 * (cap + 1) + 1));
      if (threadIdx.x < 32) {
        givens_step_warp<T>(j, cap, h1T, hT, hp, colT, gcT, gsT, gT, tol_abs, K.scal + 2, K.flags, K.scal);
      } else {
        for (int q = threadIdx.x - 32; q < nown; q += NT - 32) {
          const size_t e = on(q);
          const cx<T> w = sub_comb<T>(Wt[q], nv, hT, OwnBasis<T>{Vs, V, vstride, q, nres, n, e});
          Wt[q] = w;
          wbuf[e] = w;
        }
      }
      vec_units += 2 * nv + (nv + 1);
    }
    s = hp > 0 ? T(1) / sqrt(T(hp)) : T(0);
    src = wbuf;
    flag_raise(nflag, bid, (unsigned)(j + 1));  // ends with the CTA barrier the rotation needs too
    if (bid == 0) {  // CTA 0 keeps the rotated column j (FP64) for the final triangular solve
      double* Rc = Rg + 2 * (size_t)j * (cap + 1);
      for (int i = threadIdx.x; i < 2 * nv; i += NT) Rc[i] = double(colT[i]);
    }
    est = K.scal[2];
    if (K.flags[0]) {
      jstop = j + 1;
      break;
    }
  }
  // y = R^-1 g by warp 0 of CTA 0 (after the barrier that makes the last column of R visible
  // to warp 0), then x += V y at the own nodes
  __syncthreads();
  double* y = Rg + 2 * (size_t)cap * (cap + 1);
  if (bid == 0 && threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double* gw = K.h;
    double* dinv = K.h1;
    for (int i = lane; i < 2 * jstop; i += 32) gw[i] = double(gT[i]);
    for (int i = lane; i < jstop; i += 32) {
      const double dr = Rg[2 * ((size_t)i * (cap + 1) + i)], di = Rg[2 * ((size_t)i * (cap + 1) + i) + 1];
      const double d = dr * dr + di * di;
      dinv[2 * i] = dr / d;
      dinv[2 * i + 1] = -di / d;
    }
    __syncwarp();
    for (int i = jstop - 1; i >= 0; --i) {
      const double* Ri = Rg + 2 * (size_t)i * (cap + 1);
      double yr = 0, yi = 0;
      if (lane == 0) {
        const double sr = gw[2 * i], si = gw[2 * i + 1];
        const double ir = dinv[2 * i], ii = dinv[2 * i + 1];
        yr = sr * ir - si * ii;
        yi = sr * ii + si * ir;
        y[2 * i] = yr;
        y[2 * i + 1] = yi;
      }
      yr = __shfl_sync(0xffffffffu, yr, 0);
      yi = __shfl_sync(0xffffffffu, yi, 0);
      for (int k = lane; k < i; k += 32) {
        const double rr = Ri[2 * k], ri = Ri[2 * k + 1];
        gw[2 * k] -= rr * yr - ri * yi;
        gw[2 * k + 1] -= rr * yi + ri * yr;
      }
      __syncwarp();
    }
  }
  if (bid == 0 && threadIdx.x == 0) {
    st->its = jstop;
    st->est = est;
    st->total_its += jstop;
    st->total_reorth += reorths;
    st->total_bytes += (vec_units + jstop + 2) * eb * (double)n + k_units * ekb * (double)n;
  }
  if (!grid_sync(st, G)) return;
  for (int i = threadIdx.x; i < 2 * jstop; i += NT) sc[i] = T(-__ldcg(y + i));
  __syncthreads();
  // x + V y as x - V (-y): the combination routine with negated coefficients
  for (int q = threadIdx.x; q < nown; q += NT) {
    const size_t e = on(q);
    x[e] = sub_comb<T>(x[e], jstop, sc, OwnBasis<T>{Vs, V, vstride, q, nres, n, e});
  }
  timing_end(st, G);
}

template <typename T>
OpP<T> mkop(const hz::OpDesc& d) {
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
size_t krylov_smem_bytes(int cap) {
  return sizeof(double) * (2 * (2 * (cap + 1) + 2) + cap + 2 * cap + 2 * (cap + 1) + kWred + 4) + sizeof(int) * 4 +
         sizeof(T) * (8 * (cap + 1) + 4) + 64;
}

template <typename T, int R, int TS = 0>
size_t kshared_bytes(int cap) {
  const size_t tile = tile_smem_bytes<T, R>(TileShape<TS>::X, TileShape<TS>::Y);
  const size_t region = (sizeof(T) == 4 && kRingBytes > tile) ? kRingBytes : tile;
  return region + krylov_smem_bytes<T>(cap);
}

// Shared memory of the tile-owned form: tile, own z / w, nres own basis vectors, Krylov scratch.
template <typename T, int R>
size_t tile_form_smem(int TX, int TY, int cap, int nres = 0) {
  const size_t vs = (size_t)(TX + 1) * (TY + 1);
  return tile_smem_bytes<T, R>(TX + 1, TY + 1) + sizeof(cx<T>) * vs * (1 + (size_t)nres) + krylov_smem_bytes<T>(cap);
}

// Basis vectors of the own nodes that the tile-owned form keeps in shared memory: as many as fit
// (at most cap + 1) while every tile stays co-resident.
template <typename T, int R>
int tile_form_nres(int nx, int ny, int cap, int TX, int TY) {
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  const size_t base = tile_form_smem<T, R>(TX, TY, cap, 0);
  const size_t per_vec = sizeof(cx<T>) * (size_t)(TX + 1) * (TY + 1);
  if (base > (size_t)optin) return 0;
  int nres = (int)std::min<size_t>((size_t)cap + 1, ((size_t)optin - base) / per_vec);
  const int tiles = tiles_along(nx, TX) * tiles_along(ny, TY);
  for (; nres > 0; nres = nres > 8 ? nres - 8 : 0) {
    const size_t sm = tile_form_smem<T, R>(TX, TY, cap, nres);
    int per = 0;
    if (hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_gmres_tile2<T, R>), sm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gmres_tile2<T, R>, NT, sm) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (tiles <= per * sms) break;
  }
  return nres;
}

// Tile shapes of the tile-owned form that fit an nx x ny level: every CTA owns one tile and all
// tiles are co-resident.  Written most tiles first (one shape per tile count, the larger tile on
// a tie); returns how many were written (at most maxc).
template <typename T, int R>
int tile_form_list(int nx, int ny, int cap, int* TXo, int* TYo, int maxc) {
  static const int cand[4][2] = {{64, 32}, {32, 32}, {32, 16}, {16, 16}};
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  int m = 0, cnt[4];
  for (const auto& c : cand) {
    const int TX = c[0], TY = c[1];
    const size_t sm = tile_form_smem<T, R>(TX, TY, cap);
    if (sm > (size_t)optin) continue;
    const int nt = tiles_along(nx, TX) * tiles_along(ny, TY);
    if (hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_gmres_tile2<T, R>), sm) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gmres_tile2<T, R>, NT, sm) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (nt > per * sms) continue;
    bool dup = false;
    for (int i = 0; i < m; ++i) dup |= cnt[i] == nt;
    if (dup || m == maxc) continue;
    int i = m++;
    for (; i > 0 && cnt[i - 1] < nt; --i) {  // insertion by decreasing tile count
      cnt[i] = cnt[i - 1];
      TXo[i] = TXo[i - 1];
      TYo[i] = TYo[i - 1];
    }
    cnt[i] = nt;
    TXo[i] = TX;
    TYo[i] = TY;
  }
  return m;
}

// Default tile shape of the tile-owned form: the fitting shape with the most tiles.  Returns the
// tile count (0: the form does not fit this level).
template <typename T, int R>
int tile_form_choice(int nx, int ny, int cap, int* TXo, int* TYo) {
  int tx[4], ty[4];
  if (tile_form_list<T, R>(nx, ny, cap, tx, ty, 4) == 0) return 0;
  *TXo = tx[0];
  *TYo = ty[0];
  return tiles_along(nx, tx[0]) * tiles_along(ny, ty[0]);
}

template <typename T, int R>
cudaError_t gmres_tile_t(hz::Ctx& c, const hz::OpDesc& d, const void* b, void* x, void* V, void* w0,
                         unsigned* nflag, double* partA, double* partB, double* Rg, hz::GmresState* st, int cap,
                         double tol, int TX, int TY, double eta2) {
  TileGrid tg;
  tg.TX = TX;
  tg.TY = TY;
  tg.ntx = tiles_along(d.nx, TX);
  tg.nty = tiles_along(d.ny, TY);
  const int grid = tg.ntx * tg.nty;
  // resident basis vectors, decided once per level shape and process
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, int> nres_cache;
  int nres;
  {
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(d.nx, d.ny, cap, TX, TY);
    auto it = nres_cache.find(key);
    if (it == nres_cache.end()) it = nres_cache.emplace(key, tile_form_nres<T, R>(d.nx, d.ny, cap, TX, TY)).first;
    nres = it->second;
  }
  const size_t sm = tile_form_smem<T, R>(TX, TY, cap, nres);
  cudaError_t e = hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_gmres_tile2<T, R>), sm);
  if (e != cudaSuccess) return e;
  OpP<T> P = mkop<T>(d);
  const cx<T>* bb = reinterpret_cast<const cx<T>*>(b);
  cx<T>* xx = reinterpret_cast<cx<T>*>(x);
  cx<T>* VV = reinterpret_cast<cx<T>*>(V);
  cx<T>* wb = reinterpret_cast<cx<T>*>(w0);
  void* args[] = {&P, &tg, &bb, &xx, &VV, &wb, &nflag, &partA, &partB, &Rg, &st, &cap, &nres, &tol, &eta2};
  hz::ProfScope ps(c, hz::F_GMRES, 0.0);
  return cudaLaunchCooperativeKernel((const void*)k_gmres_tile2<T, R>, dim3(grid), dim3(NT), args, sm, c.s);
}

// The grid form uses 64 x 32 tiles on FP32 levels of at least 2^18 nodes with the radius-3
// coarse stencil, 32 x 16 tiles otherwise.
template <typename T, int R>
constexpr bool kHasWide = sizeof(T) == 4 && R == 3;
template <typename T, int R>
constexpr bool wide_tiles(size_t n) {
  return kHasWide<T, R> && n >= ((size_t)1 << 18);
}

template <typename T, int R>
cudaError_t gmres_t(hz::Ctx& c, const hz::OpDesc& d, const void* b, void* x, void* V, void* w0, void* w1,
                    double* partA, double* partB, int pstride, double* Rg, hz::GmresState* st, int cap, double tol,
                    int grid, bool cluster, int nrhs, double eta2) {
  const size_t sm = kshared_bytes<T, R>(cap);
  OpP<T> P = mkop<T>(d);
  const cx<T>* bb = reinterpret_cast<const cx<T>*>(b);
  cx<T>* xx = reinterpret_cast<cx<T>*>(x);
  cx<T>* VV = reinterpret_cast<cx<T>*>(V);
  cx<T>* a0 = reinterpret_cast<cx<T>*>(w0);
  cx<T>* a1 = reinterpret_cast<cx<T>*>(w1);
  if (cluster) {  // nrhs clusters of `grid` CTAs, cluster q solves right-hand side q
    if (grid < 1 || grid > kMaxCluster || nrhs < 1) return cudaErrorInvalidValue;
    cudaError_t e = hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_gmres<T, R, true>), sm);
    if (e != cudaSuccess) return e;
    if (grid > 8 && (e = cudaFuncSetAttribute(k_gmres<T, R, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
                        cudaSuccess)
      return e;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid * nrhs);
    lc.blockDim = dim3(NT);
    lc.dynamicSmemBytes = sm;
    lc.stream = c.s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = grid;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    hz::ProfScope ps(c, hz::F_GMRES, 0.0);
    return cudaLaunchKernelEx(&lc, k_gmres<T, R, true>, P, bb, xx, VV, a0, a1, partA, partB, pstride, Rg, st, cap, tol,
                              eta2);
  }
  if (nrhs != 1) return cudaErrorInvalidValue;  // the cooperative grid solves one right-hand side
  void* args[] = {&P, &bb, &xx, &VV, &a0, &a1, &partA, &partB, &pstride, &Rg, &st, &cap, &tol, &eta2};
  if constexpr (kHasWide<T, R>) {
    if (wide_tiles<T, R>((size_t)d.nx * d.ny)) {
      const size_t smw = kshared_bytes<T, R, 1>(cap);
      cudaError_t e = hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_gmres<T, R, false, 1>), smw);
      if (e != cudaSuccess) return e;
      hz::ProfScope ps(c, hz::F_GMRES, 0.0);
      return cudaLaunchCooperativeKernel((const void*)k_gmres<T, R, false, 1>, dim3(grid), dim3(NT), args, smw, c.s);
    }
  }
  cudaError_t e = hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_gmres<T, R, false>), sm);
  if (e != cudaSuccess) return e;
  hz::ProfScope ps(c, hz::F_GMRES, 0.0);
  return cudaLaunchCooperativeKernel((const void*)k_gmres<T, R, false>, dim3(grid), dim3(NT), args, sm, c.s);
}

// Largest cluster (16, else 8) of the cluster form that the device can place, 0 if none.
template <typename T, int R>
int cluster_size_t(int cap) {
  const size_t sm = kshared_bytes<T, R>(cap);
  if (hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_gmres<T, R, true>), sm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const bool np = cudaFuncSetAttribute(k_gmres<T, R, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess;
  cudaGetLastError();
  for (int C = np ? kMaxCluster : 8; C >= 8; C /= 2) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(C);
    lc.blockDim = dim3(NT);
    lc.dynamicSmemBytes = sm;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, k_gmres<T, R, true>, &lc) == cudaSuccess && num >= 1) return C;
    cudaGetLastError();
  }
  return 0;
}

template <typename T, int R>
int max_grid_t(int cap, size_t n) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if constexpr (kHasWide<T, R>) {
    if (wide_tiles<T, R>(n)) {
      const size_t smw = kshared_bytes<T, R, 1>(cap);
      if (hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_gmres<T, R, false, 1>), smw) != cudaSuccess) return 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gmres<T, R, false, 1>, NT, smw) != cudaSuccess)
        return 0;
      return per * sms;
    }
  }
  const size_t sm = kshared_bytes<T, R>(cap);
  if (hz::ensure_dyn_smem(reinterpret_cast<const void*>(k_gmres<T, R, false>), sm) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gmres<T, R, false>, NT, sm) != cudaSuccess) return 0;
  return per * sms;
}

}  // namespace

namespace hz {

int gmres_max_grid(int dt, int R, int cap, size_t n) {
  if (dt == C128) {
    if (R == 1) return max_grid_t<double, 1>(cap, n);
    if (R == 2) return max_grid_t<double, 2>(cap, n);
    if (R == 3) return max_grid_t<double, 3>(cap, n);
  } else {
    if (R == 1) return max_grid_t<float, 1>(cap, n);
    if (R == 2) return max_grid_t<float, 2>(cap, n);
    if (R == 3) return max_grid_t<float, 3>(cap, n);
  }
  return 0;
}

int gmres_cluster_size(int dt, int R, int cap) {
  if (dt == C128) {
    if (R == 1) return cluster_size_t<double, 1>(cap);
    if (R == 2) return cluster_size_t<double, 2>(cap);
    if (R == 3) return cluster_size_t<double, 3>(cap);
  } else {
    if (R == 1) return cluster_size_t<float, 1>(cap);
    if (R == 2) return cluster_size_t<float, 2>(cap);
    if (R == 3) return cluster_size_t<float, 3>(cap);
  }
  return 0;
}

// The tile-owned form runs with FP32 vectors only (FP64 tiles would not fit the registers).
int gmres_tile_form(int dt, int R, int nx, int ny, int cap, int* TX, int* TY) {
  if (dt != C64) return 0;
  if (R == 1) return tile_form_choice<float, 1>(nx, ny, cap, TX, TY);
  if (R == 2) return tile_form_choice<float, 2>(nx, ny, cap, TX, TY);
  if (R == 3) return tile_form_choice<float, 3>(nx, ny, cap, TX, TY);
  return 0;
}

int gmres_tile_forms(int dt, int R, int nx, int ny, int cap, int* TX, int* TY, int maxc) {
  if (dt != C64) return 0;
  if (R == 1) return tile_form_list<float, 1>(nx, ny, cap, TX, TY, maxc);
  if (R == 2) return tile_form_list<float, 2>(nx, ny, cap, TX, TY, maxc);
  if (R == 3) return tile_form_list<float, 3>(nx, ny, cap, TX, TY, maxc);
  return 0;
}

cudaError_t launch_gmres_tile(Ctx& c, const OpDesc& M, int dt, const void* b, void* x, void* V, void* w0,
                              unsigned* nflag, double* partA, double* partB, double* Rg, GmresState* st, int cap,
                              double tol, int TX, int TY, double eta2) {
#define HZ_GT(T_, R_) return gmres_tile_t<T_, R_>(c, M, b, x, V, w0, nflag, partA, partB, Rg, st, cap, tol, TX, TY, eta2)
  if (dt == C64) {
    if (M.R == 1) HZ_GT(float, 1);
    if (M.R == 2) HZ_GT(float, 2);
    if (M.R == 3) HZ_GT(float, 3);
  }
#undef HZ_GT
  return cudaErrorInvalidValue;
}

cudaError_t launch_gmres_persistent(Ctx& c, const OpDesc& M, int dt, const void* b, void* x, void* V, void* w0,
                                    void* w1, double* partA, double* partB, int pstride, double* Rg, GmresState* st,
                                    int cap, double tol, int grid, bool cluster, int nrhs, double eta2) {
#define HZ_GM(T_, R_) \
  return gmres_t<T_, R_>(c, M, b, x, V, w0, w1, partA, partB, pstride, Rg, st, cap, tol, grid, cluster, nrhs, eta2)
  if (dt == C128) {
    if (M.R == 1) HZ_GM(double, 1);
    if (M.R == 2) HZ_GM(double, 2);
    if (M.R == 3) HZ_GM(double, 3);
  } else {
    if (M.R == 1) HZ_GM(float, 1);
    if (M.R == 2) HZ_GM(float, 2);
    if (M.R == 3) HZ_GM(float, 3);
  }
#undef HZ_GM
  return cudaErrorInvalidValue;
}

}  // namespace hz
