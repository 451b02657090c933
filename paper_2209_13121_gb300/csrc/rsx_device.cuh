// Device-side building blocks of the GB300 P-RSoXS path: complex helpers
// and the shared-memory Stockham FFT used by the x and y (and z) passes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rsx {

template <typename R> struct RT;
template <> struct RT<float> {
  using C = float2;
  using V4 = float4;
  static __host__ __device__ __forceinline__ C mk(float a, float b) { return make_float2(a, b); }
};
template <> struct RT<double> {
  using C = double2;
  using V4 = double4_32a;  // 32-byte Real4 of the double build (Sec. 4.1)
  static __host__ __device__ __forceinline__ C mk(double a, double b) { return make_double2(a, b); }
};

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// multiply by -i
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
template <typename C, typename R> __device__ __forceinline__ R cnorm2(C a) { return a.x * a.x + a.y * a.y; }

// ---------------------------------------------------------------------------
// Shared-memory Stockham FFT (forward, unnormalised).
//
// `nfft` independent transforms of length N = 2^logN live in shared memory
// at buf[f * fstride + i * estride].  A radix-RAD pass with span Ns (the
// product of the radices already applied) takes butterfly j of transform f,
//   v_r = x[j + r N/RAD] * W_N^(r k N/(RAD Ns)),  k = j mod Ns,
// applies the RAD-point DFT and writes y[(j - k) RAD + k + r Ns] = V_r; after
// log passes the result is in natural order (self-sorting).  One radix-2 pass
// precedes the radix-4 passes when logN is odd.  tw[t] = exp(-2 pi i t / N).
//
// Each pass reads all its inputs into registers, synchronises, then writes,
// so one buffer serves as both source and destination.  Items are spread
// over the block's T threads, at most MAXI per thread.  F_FAST picks the
// item order: consecutive threads take consecutive transforms (column
// transforms, contiguous in f) or consecutive butterflies (row transforms).
// ---------------------------------------------------------------------------
template <typename R, int RAD, int MAXI, bool F_FAST>
__device__ __forceinline__ void stockham_pass(typename RT<R>::C* buf, int logN, int logNs, int nfft,
                                              int lognfft, int fstride, int estride,
                                              const typename RT<R>::C* tw) {
  using C = typename RT<R>::C;
  constexpr int LOGRAD = RAD == 2 ? 1 : 2;
  const int lognb = logN - LOGRAD;  // butterflies per transform = N / RAD
  const int nb = 1 << lognb;
  const int total = nfft << lognb;
  const int Ns = 1 << logNs;
  const int twshift = logN - LOGRAD - logNs;  // N / (RAD Ns) = 2^twshift
  C v[MAXI][RAD];
  int off[MAXI];
#pragma unroll
  for (int it = 0; it < MAXI; ++it) {
    const int item = threadIdx.x + it * blockDim.x;
    off[it] = -1;
    if (item < total) {
      int f, j;
      if (F_FAST) {
        f = lognfft >= 0 ? (item & (nfft - 1)) : (item % nfft);
        j = lognfft >= 0 ? (item >> lognfft) : (item / nfft);
      } else {
        f = item >> lognb;
        j = item & (nb - 1);
      }
      const int k = j & (Ns - 1);
      C* base = buf + (size_t)f * fstride;
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[it][r] = base[(j + r * nb) * estride];
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[it][r] = cmul(v[it][r], tw[(r * k) << twshift]);
      if (RAD == 2) {
        C a = v[it][0], b = v[it][1];
        v[it][0] = cadd(a, b);
        v[it][1] = csub(a, b);
      } else {
        C a0 = cadd(v[it][0], v[it][2]);
        C a1 = csub(v[it][0], v[it][2]);
        C a2 = cadd(v[it][1], v[it][3]);
        C a3 = cmul_mi(csub(v[it][1], v[it][3]));
        v[it][0] = cadd(a0, a2);
        v[it][1] = cadd(a1, a3);
        v[it][2] = csub(a0, a2);
        v[it][3] = csub(a1, a3);
      }
      off[it] = f * fstride + (((j - k) << LOGRAD) + k) * estride;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < MAXI; ++it) {
    if (off[it] >= 0) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) buf[off[it] + r * Ns * estride] = v[it][r];
    }
  }
  __syncthreads();
}

// Whole transform: nfft transforms of length 2^logN.  The caller has
// synchronised after filling buf and tw; on return buf holds the spectra
// and the block is synchronised.  lognfft < 0 when nfft is not a power of 2
// (only allowed with F_FAST = false).
template <typename R, int MAXI4, int MAXI2, bool F_FAST>
__device__ __forceinline__ void block_fft(typename RT<R>::C* buf, int logN, int nfft, int lognfft,
                                          int fstride, int estride, const typename RT<R>::C* tw) {
  int logNs = 0;
  if (logN & 1) {
    stockham_pass<R, 2, MAXI2, F_FAST>(buf, logN, 0, nfft, lognfft, fstride, estride, tw);
    logNs = 1;
  }
  for (; logNs < logN; logNs += 2)
    stockham_pass<R, 4, MAXI4, F_FAST>(buf, logN, logNs, nfft, lognfft, fstride, estride, tw);
}

}  // namespace rsx
