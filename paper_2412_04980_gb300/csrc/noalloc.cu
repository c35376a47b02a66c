// hz_true_residual_noalloc: the relative residual ||b - A_h u|| / ||b|| of each right-hand
// side, computed without allocating any device memory.
//
// Who needs it: callers that cannot call cudaMalloc (or any allocating library routine)
// at the point where they check a solution -- for example a plugin whose host
// application owns and budgets every device allocation, or a real-time loop that must
// not enter the allocator.  hz_solve computes the same quantity with a residual vector
// and reduction workspace that the handle allocated; this entry point fuses the 5-point
// residual with the norms and keeps its block partial sums in a fixed static array.
//
// Scratch: g_partials, a file-scope __device__ array of 1216 x 2 x 64 doubles
// (1216 CTAs x 2 sums x HZ_NOALLOC_MAX_RHS right-hand sides, 1.25 MB).  Every GPU on which
// a handle was set up holds it until the process exits.  Host code cannot use the array's
// name as a device address, so hz_setup looks the address up with cudaGetSymbolAddress on
// the handle's device and queries both kernels' attributes there: with CUDA's lazy module
// loading that is the moment the module (kernels and array) is loaded, so the array is
// reserved during hz_setup and no call of this entry point, the first included, reserves
// device memory.  Every call reuses the same array and each partial is written before it is
// read, so nothing needs clearing; calls that overlap on the GPU (concurrent streams,
// several host threads, several handles) race on the array and must be serialised.
#include <mutex>
#include <string>

#include "hz_core.h"
#include "hz_device.cuh"

using namespace hzd;

namespace {

constexpr int kParts = 1216;
constexpr int kMaxRhs = 64;
constexpr int kNT = 256;
static __device__ __align__(256) double g_partials[kParts * 2 * kMaxRhs];

// partial sums of |b - A u|^2 and |b|^2, Sommerfeld 5-point rows with ghost points
__global__ void __launch_bounds__(kNT) k_resid_norm(int nx, int ny, double c, double H, const double* __restrict__ k,
                                                    const cx<double>* __restrict__ b, const cx<double>* __restrict__ u,
                                                    double* __restrict__ part, int bc, size_t kstride) {
  __shared__ double sr[kNT / 32], sb[kNT / 32];
  const size_t n = (size_t)nx * ny;
  const size_t off = (size_t)blockIdx.y * n;
  k += blockIdx.y * kstride;  // per-right-hand-side wavenumber fields (kstride 0: shared)
  double r2 = 0, b2 = 0;
  for (size_t i = blockIdx.x * (size_t)kNT + threadIdx.x; i < n; i += (size_t)gridDim.x * kNT) {
    const int gy = (int)(i / nx), gx = (int)(i - (size_t)gy * nx);
    const cx<double> uc = u[off + i];
    const double kk = k[i];
    // neighbour values with the ghost point u_out = u_in + 2 H i k_b u_b substituted
    auto nb = [&](int x, int y, int xi, int yi) -> cx<double> {
      if (x >= 0 && x < nx && y >= 0 && y < ny) return u[off + (size_t)y * nx + x];
      if (bc != 0) return mk<double>(0.0, 0.0);
      cx<double> ui = u[off + (size_t)yi * nx + xi];
      const double t = 2.0 * H * kk;
      return mk<double>(ui.re - t * uc.im, ui.im + t * uc.re);
    };
    cx<double> s = (nb(gx + 1, gy, gx - 1, gy) + nb(gx - 1, gy, gx + 1, gy)) +
                   (nb(gx, gy + 1, gx, gy - 1) + nb(gx, gy - 1, gx, gy + 1));
    cx<double> au = mk<double>(c * (4.0 * uc.re - s.re) - kk * kk * uc.re, c * (4.0 * uc.im - s.im) - kk * kk * uc.im);
    cx<double> bv = b[off + i];
    cx<double> r = bv - au;
    r2 += r.re * r.re + r.im * r.im;
    b2 += bv.re * bv.re + bv.im * bv.im;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    b2 += __shfl_xor_sync(0xffffffffu, b2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = r2;
    sb[threadIdx.x >> 5] = b2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, q = 0;
    for (int w = 0; w < kNT / 32; ++w) {
      a += sr[w];
      q += sb[w];
    }
    part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 2] = a;
    part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 2 + 1] = q;
  }
}

// out[rhs] = sqrt(sum |r|^2 / sum |b|^2) (sqrt(sum |r|^2) when b = 0), fixed summation order
__global__ void __launch_bounds__(kNT) k_resid_finish(const double* __restrict__ part, int nparts,
                                                      double* __restrict__ out) {
  __shared__ double sr[kNT / 32], sb[kNT / 32];
  const double* p = part + (size_t)blockIdx.x * nparts * 2;
  double r2 = 0, b2 = 0;
  for (int i = threadIdx.x; i < nparts; i += kNT) {
    r2 += p[2 * i];
    b2 += p[2 * i + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    b2 += __shfl_xor_sync(0xffffffffu, b2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = r2;
    sb[threadIdx.x >> 5] = b2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, q = 0;
    for (int w = 0; w < kNT / 32; ++w) {
      a += sr[w];
      q += sb[w];
    }
    out[blockIdx.x] = q > 0 ? sqrt(a / q) : sqrt(a);
  }
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
double* g_addr[kMaxDevices] = {};

// Device address of g_partials on device dev (looked up once per device, with dev current).
int scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    hz::set_error("device index beyond the static scratch table");
    return HZ_ENOTSUP;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) return hz::status_of(e, "cudaGetSymbolAddress(g_partials)");
    g_addr[dev] = reinterpret_cast<double*>(p);
  }
  *out = g_addr[dev];
  return HZ_OK;
}

}  // namespace

namespace hz {

// Called by setup() with the handle's device current: loads this file's module (kernels and
// the static array) and caches the array's device address.
int noalloc_prepare(Handle* H) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_resid_norm);
  if (e != cudaSuccess) return status_of(e, "cudaFuncGetAttributes(k_resid_norm)");
  e = cudaFuncGetAttributes(&fa, k_resid_finish);
  if (e != cudaSuccess) return status_of(e, "cudaFuncGetAttributes(k_resid_finish)");
  double* part = nullptr;
  return scratch_address(H->device, &part);
}

}  // namespace hz

using namespace hz;

struct hz_handle_s {
  Handle h;
};

extern "C" int hz_true_residual_noalloc(hz_handle hp, const void* b, const void* u, int nrhs, double* relres_dev) {
  if (!hp || !b || !u || !relres_dev) {
    hz::set_error("null argument");
    return HZ_EINVAL;
  }
  if (nrhs < 1 || nrhs > kMaxRhs) {
    hz::set_error("nrhs must be in [1, HZ_NOALLOC_MAX_RHS]");
    return HZ_EINVAL;
  }
  hz::Handle* H = &hp->h;
  if (H->cfg.per_rhs_k && nrhs > H->nbmax) {
    hz::set_error("with per_rhs_k every right-hand side needs its own wavenumber field: nrhs <= max_rhs");
    return HZ_EINVAL;
  }
  // an error left by earlier, unrelated work is reported as such, not as this call's failure
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    hz::set_error(std::string("a CUDA error was pending before hz_true_residual_noalloc: ") + cudaGetErrorString(e));
    return HZ_ECUDA;
  }
  int dev = -1;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hz::status_of(e, "cudaGetDevice");
  if (dev != H->device) {
    hz::set_error("the current CUDA device is not the device the handle was set up on");
    return HZ_EINVAL;
  }
  const hz::Level& L = H->lv[0];
  double* part = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    part = g_addr[dev];  // set by hz_setup on this device
  }
  if (!part) {
    hz::set_error("the static scratch array was not prepared on this device");
    return HZ_ENOTSUP;
  }
  const size_t n = L.n;
  size_t nb = (n + kNT * 4 - 1) / (kNT * 4);
  const int nparts = (int)(nb < kParts ? (nb > 0 ? nb : 1) : kParts);
  k_resid_norm<<<dim3(nparts, nrhs), kNT, 0, H->ctx.s>>>(L.nx, L.ny, 1.0 / (H->g.h * H->g.h), H->g.h, L.k_d,
                                                         reinterpret_cast<const cx<double>*>(b),
                                                         reinterpret_cast<const cx<double>*>(u), part, H->g.bc,
                                                         L.kstride);
  e = cudaGetLastError();
  if (e != cudaSuccess) return hz::status_of(e, "k_resid_norm");
  k_resid_finish<<<nrhs, kNT, 0, H->ctx.s>>>(part, nparts, relres_dev);
  e = cudaGetLastError();
  return e == cudaSuccess ? HZ_OK : hz::status_of(e, "k_resid_finish");
}
