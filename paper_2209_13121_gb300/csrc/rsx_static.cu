// rsx_scatter_angle_noalloc: one angle of the hot path without any device
// allocation, for callers that cannot call cudaMalloc (for example code
// running inside another framework's memory pool or allocator-free
// embedded hosts).  Its working memory is a fixed array in this file.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/rsx.h"
#include "rsx_device.cuh"
#include "rsx_kernels.h"

namespace {

using rsx::Geo;
using rsx::PolParams;

constexpr long long kMaxVox = RSX_NOALLOC_MAX_VOXELS;
constexpr long long kMaxPix = RSX_NOALLOC_MAX_PIXELS;
constexpr int kMaxLen = 4096;  // nx, ny, nz limit of the twiddle tables

// Byte layout of the scratch array: p (3 N complex float), the per-pixel
// Ewald geometry, and the x, y, z twiddle tables.
constexpr size_t kOffP = 0;
constexpr size_t kBytesP = 3 * (size_t)kMaxVox * sizeof(float2);
constexpr size_t kOffGeo = kOffP + kBytesP;
constexpr size_t kBytesGeo = (size_t)kMaxPix * sizeof(Geo<float>);
constexpr size_t kOffTw = kOffGeo + kBytesGeo;
constexpr size_t kBytesTw = 3 * (size_t)kMaxLen * sizeof(float2);
constexpr size_t kScratchBytes = kOffTw + kBytesTw;

// Held by every GPU that loads this library, until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, set once per device.
std::mutex g_mu;
void* g_addr[128] = {nullptr};

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  rsx::set_last_error(buf);
  return code;
}

bool is_pow2(long long n) { return n >= 1 && (n & (n - 1)) == 0; }

// exp(-2 pi i t / n) in float, from the double-precision sincospi.
__global__ void k_twiddle_f32(float2* tw, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double s, c;
  sincospi(-2.0 * (double)t / (double)n, &s, &c);
  tw[t] = make_float2((float)c, (float)s);
}

int scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(RSX_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 128) return fail(RSX_ERR_UNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return fail(RSX_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return RSX_OK;
}

}  // namespace

int rsx_scatter_angle_noalloc(const void* M, int nx, int ny, int nz, int n_components,
                              double voxel_nm, double energy_ev, const double* constants,
                              double alpha_rad, int frame, void* img_out, void* stream) {
  if (!M || !constants || !img_out) return fail(RSX_ERR_INVALID, "NULL argument");
  if (!is_pow2(nx) || nx > kMaxLen || !is_pow2(ny) || ny > kMaxLen)
    return fail(RSX_ERR_INVALID, "nx=%d, ny=%d: each must be a power of two <= %d", nx, ny, kMaxLen);
  if (nz < 1 || nz > kMaxLen) return fail(RSX_ERR_INVALID, "nz=%d outside [1, %d]", nz, kMaxLen);
  const long long N = (long long)nx * ny * nz, npix = (long long)nx * ny;
  if (N > kMaxVox || npix > kMaxPix)
    return fail(RSX_ERR_INVALID,
                "grid %dx%dx%d exceeds the fixed scratch (at most %lld voxels and %lld pixels)", nx,
                ny, nz, kMaxVox, kMaxPix);
  if (n_components < 1 || n_components > RSX_MAX_COMPONENTS)
    return fail(RSX_ERR_INVALID, "n_components=%d outside [1, %d]", n_components,
                RSX_MAX_COMPONENTS);
  if (!(voxel_nm > 0.0) || !isfinite(voxel_nm) || !(energy_ev > 0.0) || !isfinite(energy_ev) ||
      !isfinite(alpha_rad))
    return fail(RSX_ERR_INVALID, "voxel size, energy and angle must be finite, size and energy > 0");
  if (frame != RSX_FRAME_LITERAL && frame != RSX_FRAME_LAB)
    return fail(RSX_ERR_INVALID, "frame=%d", frame);
  if (((uintptr_t)M) % 16 != 0 || ((uintptr_t)img_out) % 4 != 0)
    return fail(RSX_ERR_INVALID, "M must be 16-byte aligned, img_out 4-byte aligned");
  for (int i = 0; i < 4 * n_components; ++i)
    if (!isfinite(constants[i])) return fail(RSX_ERR_INVALID, "optical constant %d not finite", i);

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(RSX_ERR_INVALID, "M and img_out must be device memory (no CUDA device)");
  }
  int rc = rsx::check_device_pointer(M, dev, "M");
  if (rc) return rc;
  if ((rc = rsx::check_device_pointer(img_out, dev, "img_out"))) return rc;

  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  char* sc = (char*)base;
  float2* p = (float2*)(sc + kOffP);
  Geo<float>* geo = (Geo<float>*)(sc + kOffGeo);
  float2* twx = (float2*)(sc + kOffTw);
  float2* twy = twx + kMaxLen;
  float2* twz = twy + kMaxLen;
  cudaStream_t s = (cudaStream_t)stream;

  // Same per-energy constants as the context path: eps = n - 1 = -delta + i beta.
  PolParams<float> pp;
  memset(&pp, 0, sizeof(pp));
  for (int j = 0; j < n_components; ++j) {
    const double* k = constants + 4 * j;
    const double epr = -k[0], epi = k[1], eqr = -k[2], eqi = k[3];
    const double tr = (epr + 2.0 * eqr) / 3.0, ti = (epi + 2.0 * eqi) / 3.0;
    rsx::set_component(pp, j, tr, ti, eqr - tr, eqi - ti, epr - eqr, epi - eqi);
  }
  pp.ce = (float)cos(alpha_rad);
  pp.se = (float)sin(alpha_rad);
  pp.c = n_components;
  pp.literal = frame == RSX_FRAME_LITERAL;
  pp.add_ref = 0;
  const double pi = 3.14159265358979323846;
  const double k_in = 2.0 * pi / (1239.84198 / energy_ev);
  const double ref = -(double)(n_components - 1) / (4.0 * pi) * (double)N;
  float dc[3] = {(float)ref, 0.f, 0.f};
  if (!pp.literal) {
    dc[0] = (float)(ref * cos(alpha_rad));
    dc[1] = (float)(ref * sin(alpha_rad));
  }

  cudaError_t e;
  const int lens[3] = {nx, ny, nz};
  float2* tws[3] = {twx, twy, twz};
  for (int a = 0; a < 3; ++a) {
    k_twiddle_f32<<<(lens[a] + 255) / 256, 256, 0, s>>>(tws[a], lens[a]);
    if ((e = cudaGetLastError()) != cudaSuccess)
      return fail(RSX_ERR_CUDA, "twiddle kernel: %s", cudaGetErrorString(e));
  }
  if ((e = rsx::launch_geometry<float>(geo, nx, ny, nz, voxel_nm, k_in, s)) != cudaSuccess)
    return fail(RSX_ERR_CUDA, "geometry kernel: %s", cudaGetErrorString(e));
  if ((e = rsx::launch_pol_fftx<float>(M, nx, ny, nz, pp, true, p, twx, s)) != cudaSuccess)
    return fail(RSX_ERR_CUDA, "polarisation + x-FFT kernel: %s", cudaGetErrorString(e));
  if ((e = rsx::launch_col_fft<float>(p, ny, nx, nx, {3LL * nz, nz, N, npix, 0}, twy, s)) !=
      cudaSuccess)
    return fail(RSX_ERR_CUDA, "y-FFT kernel: %s", cudaGetErrorString(e));
  if ((e = rsx::launch_ewald<float>(p, nx, ny, nz, geo, twz, true, dc, img_out, s)) != cudaSuccess)
    return fail(RSX_ERR_CUDA, "Ewald kernel: %s", cudaGetErrorString(e));
  return RSX_OK;
}
