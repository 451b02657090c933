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

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C> __host__ __device__ __forceinline__ C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

// Asynchronous global -> shared copies of one complex element (cp.async):
// the copy goes straight to shared memory without passing through
// registers, so a thread can keep many of them in flight.
__device__ __forceinline__ void cp_async_elem(float2* dst, const float2* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2* dst, const double2* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// Two adjacent complex floats (16 bytes, both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async_pair(float2* dst, const float2* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Wait until at most N of this thread's committed groups are still in flight.
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ---- bulk asynchronous copies (TMA, 1-D) completing on an mbarrier -------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
// Makes barrier initialisation and earlier generic-proxy accesses of shared
// memory visible to the asynchronous (bulk copy) proxy.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// tiled tensor copy (TMA) of one box at coordinates (x, y, z) -> shared
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the barrier, giving up after `limit` polls
// (each poll may suspend the thread for a hardware-defined interval).
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// OR-reduction barrier over the first n threads of the block on named
// barrier `id` (n a multiple of 32): every participant gets the OR of pred.
__device__ __forceinline__ bool named_bar_or(int id, int n, bool pred) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void named_bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned limit) {
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Shared-memory padding: one spare element after every 16, which makes the
// Stockham reads and writes below free of bank conflicts for 8- and
// 16-byte elements (checked by enumerating the warp access patterns).
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded(int n) { return n + (n >> 4) + 1; }

// ------------------------------------------------ in-register small DFTs
// a * exp(-2 pi i E / 16) for a compile-time E.
template <int E, typename C> __host__ __device__ __forceinline__ C w16(C a) {
  using R = decltype(a.x);
  constexpr int e = E & 15;
  constexpr double h = 0.70710678118654752440;
  constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173;
  if constexpr (e == 0) return a;
  else if constexpr (e == 4) return cmul_mi(a);
  else if constexpr (e == 8) { a.x = -a.x; a.y = -a.y; return a; }
  else if constexpr (e == 12) { C r; r.x = -a.y; r.y = a.x; return r; }
  else if constexpr (e == 2) { C r; r.x = R(h) * (a.x + a.y); r.y = R(h) * (a.y - a.x); return r; }
  else if constexpr (e == 6) { C r; r.x = R(h) * (a.y - a.x); r.y = -R(h) * (a.x + a.y); return r; }
  else if constexpr (e == 10) { C r; r.x = -R(h) * (a.x + a.y); r.y = R(h) * (a.x - a.y); return r; }
  else if constexpr (e == 14) { C r; r.x = R(h) * (a.x - a.y); r.y = R(h) * (a.x + a.y); return r; }
  else {
    // cos and sin of 2 pi e / 16 for odd e, from cos/sin(pi/8)
    constexpr double cs[16] = {1, c1, h, s1, 0, -s1, -h, -c1, -1, -c1, -h, -s1, 0, s1, h, c1};
    constexpr double sn[16] = {0, s1, h, c1, 1, c1, h, s1, 0, -s1, -h, -c1, -1, -c1, -h, -s1};
    const R c = R(cs[e]), s = R(sn[e]);
    C r;
    r.x = a.x * c + a.y * s;
    r.y = a.y * c - a.x * s;
    return r;
  }
}

template <typename C> __host__ __device__ __forceinline__ void dft2(C& a, C& b) {
  const C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// 4-point forward DFT in place, outputs in natural order.
template <typename C> __host__ __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  const C a0 = cadd(v0, v2), a1 = csub(v0, v2);
  const C a2 = cadd(v1, v3), a3 = cmul_mi(csub(v1, v3));
  v0 = cadd(a0, a2);
  v2 = csub(a0, a2);
  v1 = cadd(a1, a3);
  v3 = csub(a1, a3);
}

// RAD-point forward DFT of v[0..RAD).  Output index r is left in register
// v[out_pos<RAD>(r)].  8 = 4 x 2 and 16 = 4 x 4 with the inner twiddles
// exp(-2 pi i m k1 / RAD) between the two stages.
template <int RAD> __host__ __device__ constexpr int out_pos(int r) {
  return RAD == 16 ? 4 * (r & 3) + (r >> 2) : RAD == 8 ? 2 * (r & 3) + (r >> 2) : r;
}

template <int RAD, typename C> __host__ __device__ __forceinline__ void dft_reg(C* v) {
  if constexpr (RAD == 2) {
    dft2(v[0], v[1]);
  } else if constexpr (RAD == 4) {
    dft4(v[0], v[1], v[2], v[3]);
  } else if constexpr (RAD == 8) {
    // n = m + 2 n1: 4-point DFTs over n1 for m = 0, 1 -> position m + 2 k1
    dft4(v[0], v[2], v[4], v[6]);
    dft4(v[1], v[3], v[5], v[7]);
    v[3] = w16<2>(v[3]);   // W8^1
    v[5] = w16<4>(v[5]);   // W8^2
    v[7] = w16<6>(v[7]);   // W8^3
    dft2(v[0], v[1]);
    dft2(v[2], v[3]);
    dft2(v[4], v[5]);
    dft2(v[6], v[7]);
  } else {
    // n = m + 4 n1: 4-point DFTs over n1 -> a_m[k1] at position m + 4 k1
    dft4(v[0], v[4], v[8], v[12]);
    dft4(v[1], v[5], v[9], v[13]);
    dft4(v[2], v[6], v[10], v[14]);
    dft4(v[3], v[7], v[11], v[15]);
    v[5] = w16<1>(v[5]);
    v[9] = w16<2>(v[9]);
    v[13] = w16<3>(v[13]);
    v[6] = w16<2>(v[6]);
    v[10] = w16<4>(v[10]);
    v[14] = w16<6>(v[14]);
    v[7] = w16<3>(v[7]);
    v[11] = w16<6>(v[11]);
    v[15] = w16<9>(v[15]);
    // 4-point DFTs over m for each k1 -> X[k1 + 4 k2] at position 4 k1 + k2
    dft4(v[0], v[1], v[2], v[3]);
    dft4(v[4], v[5], v[6], v[7]);
    dft4(v[8], v[9], v[10], v[11]);
    dft4(v[12], v[13], v[14], v[15]);
  }
}

// a * exp(-2 pi i E / 32) for a compile-time E in [0, 16).
template <int E, typename C> __host__ __device__ __forceinline__ C w32(C a) {
  using R = decltype(a.x);
  if constexpr (E % 2 == 0) {
    return w16<E / 2>(a);
  } else {
    // cos and sin of pi e / 16 for odd e
    constexpr double cs[8] = {0.98078528040323044913, 0.83146961230254523708,
                              0.55557023301960222474, 0.19509032201612826785,
                              -0.19509032201612826785, -0.55557023301960222474,
                              -0.83146961230254523708, -0.98078528040323044913};
    constexpr double sn[8] = {0.19509032201612826785, 0.55557023301960222474,
                              0.83146961230254523708, 0.98078528040323044913,
                              0.98078528040323044913, 0.83146961230254523708,
                              0.55557023301960222474, 0.19509032201612826785};
    const R c = R(cs[E / 2]), s = R(sn[E / 2]);
    C r;
    r.x = a.x * c + a.y * s;
    r.y = a.y * c - a.x * s;
    return r;
  }
}

template <int K, typename C>
__host__ __device__ __forceinline__ void dft32_combine(C* v, const C* e, const C* o) {
  if constexpr (K < 16) {
    const C t = w32<K>(o[out_pos<16>(K)]);
    v[K] = cadd(e[out_pos<16>(K)], t);
    v[K + 16] = csub(e[out_pos<16>(K)], t);
    dft32_combine<K + 1>(v, e, o);
  }
}

// 32-point forward DFT of v[0..32) in registers, natural order in and out:
// two 16-point DFTs of the even and odd samples, X[k] = E[k] + W32^k O[k],
// X[k + 16] = E[k] - W32^k O[k].
template <typename C> __host__ __device__ __forceinline__ void dft32(C* v) {
  C e[16], o[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    e[m] = v[2 * m];
    o[m] = v[2 * m + 1];
  }
  dft_reg<16>(e);
  dft_reg<16>(o);
  dft32_combine<0>(v, e, o);
}

// v[out_pos<16>(K)] *= W32^K for K = 0..15: the odd half of a 32-point DFT
// after its 16-point DFT (compile-time twiddles).
template <int K, typename C> __device__ __forceinline__ void w32_outputs(C* v) {
  if constexpr (K < 16) {
    v[out_pos<16>(K)] = w32<K>(v[out_pos<16>(K)]);
    w32_outputs<K + 1>(v);
  }
}

// A 32-point forward DFT split over a lane pair (partner = lane ^ 16): the
// lane with h = 0 holds the even samples x[2m] in v[m], the lane with h = 1
// the odd samples x[2m + 1] (m = 0..15).  Each does its 16-point DFT, the
// lane h = 1 twiddles its outputs by W32^k, and after one exchange the h = 0
// lane holds X[k] = E[k] + W32^k O[k] and the h = 1 lane X[16 + k] =
// E[k] - W32^k O[k] in r[k], k = 0..15.  All 32 lanes of the warp take part.
template <int K, typename C>
__device__ __forceinline__ void dft32_pair_step(const C* v, C* r, int h) {
  if constexpr (K < 16) {
    using R = decltype(v[0].x);
    const C mine = v[out_pos<16>(K)];
    const C tw = w32<K>(mine);
    const C pay = h ? tw : mine;  // E[k] from h = 0, W32^k O[k] from h = 1
    C other;
    other.x = __shfl_xor_sync(0xffffffffu, pay.x, 16);
    other.y = __shfl_xor_sync(0xffffffffu, pay.y, 16);
    const R sg = h ? R(-1) : R(1);
    r[K].x = other.x + sg * pay.x;  // h = 0: E + W O ; h = 1: E - W O
    r[K].y = other.y + sg * pay.y;
    dft32_pair_step<K + 1>(v, r, h);
  }
}
template <typename C> __device__ __forceinline__ void dft32_pair(C* v, C* r, int h) {
  dft_reg<16>(v);
  dft32_pair_step<0>(v, r, h);
}

// ---------------------------------------------------------------------------
// Shared-memory Stockham FFT (forward, unnormalised).
//
// `nfft` independent transforms of length N = 2^logN live in shared memory
// at buf[padi(f * fstride + i * estride)].  A radix-RAD pass with span Ns
// (the product of the radices already applied) takes butterfly j of
// transform f,
//   v_r = x[j + r N/RAD] * W_N^(r k N/(RAD Ns)),  k = j mod Ns,
// applies the RAD-point DFT and writes y[(j - k) RAD + k + r Ns] = V_r; after
// the last pass the result is in natural order (self-sorting).  Radix-16
// passes come first, one radix-8/4/2 pass takes the remainder.
// tw[t] = exp(-2 pi i t / N).
//
// Each pass reads all its inputs into registers, synchronises, then writes,
// so one buffer is both source and destination.  Butterflies are spread
// over the block's T threads (at most ELEMS / RAD of them).  F_FAST picks
// the item order: consecutive threads take consecutive transforms (column
// transforms) or consecutive butterflies of one transform (row transforms).
// ---------------------------------------------------------------------------
template <typename R, int RAD, int ELEMS, int T, bool F_FAST>
__device__ __forceinline__ void stockham_pass(typename RT<R>::C* buf, int logN, int logNs, int nfft,
                                              int lognfft, int fstride, int estride,
                                              const typename RT<R>::C* tw) {
  using C = typename RT<R>::C;
  constexpr int LOGRAD = RAD == 2 ? 1 : RAD == 4 ? 2 : RAD == 8 ? 3 : 4;
  constexpr int MAXI = (ELEMS / RAD + T - 1) / T;
  const int lognb = logN - LOGRAD;
  const int nb = 1 << lognb;
  const int total = nfft << lognb;
  const int Ns = 1 << logNs;
  const int twshift = logN - LOGRAD - logNs;
  C v[MAXI][RAD];
  int off[MAXI];
#pragma unroll
  for (int it = 0; it < MAXI; ++it) {
    const int item = threadIdx.x + it * T;
    off[it] = -1;
    if (item < total) {
      int f, j;
      if (F_FAST) {
        f = item & (nfft - 1);
        j = item >> lognfft;
      } else {
        f = item >> lognb;
        j = item & (nb - 1);
      }
      const int k = j & (Ns - 1);
      const int base = f * fstride;
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[it][r] = buf[padi(base + (j + r * nb) * estride)];
      if (logNs > 0) {
#pragma unroll
        for (int r = 1; r < RAD; ++r) v[it][r] = cmul(v[it][r], tw[(r * k) << twshift]);
      }
      dft_reg<RAD>(v[it]);
      off[it] = base + (((j - k) << LOGRAD) + k) * estride;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < MAXI; ++it) {
    if (off[it] >= 0) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) buf[padi(off[it] + r * Ns * estride)] = v[it][out_pos<RAD>(r)];
    }
  }
  __syncthreads();
}

// nfft transforms of length 2^logN (ELEMS >= nfft << logN).  The caller has
// synchronised after filling buf and tw; on return buf holds the spectra and
// the block is synchronised.  F_FAST needs nfft = 2^lognfft.
template <typename R, int ELEMS, int T, bool F_FAST>
__device__ __forceinline__ void block_fft(typename RT<R>::C* buf, int logN, int nfft, int lognfft,
                                          int fstride, int estride, const typename RT<R>::C* tw) {
  int logNs = 0;
  for (; logN - logNs >= 4; logNs += 4)
    stockham_pass<R, 16, ELEMS, T, F_FAST>(buf, logN, logNs, nfft, lognfft, fstride, estride, tw);
  switch (logN - logNs) {
    case 3:
      stockham_pass<R, 8, ELEMS, T, F_FAST>(buf, logN, logNs, nfft, lognfft, fstride, estride, tw);
      break;
    case 2:
      stockham_pass<R, 4, ELEMS, T, F_FAST>(buf, logN, logNs, nfft, lognfft, fstride, estride, tw);
      break;
    case 1:
      stockham_pass<R, 2, ELEMS, T, F_FAST>(buf, logN, logNs, nfft, lognfft, fstride, estride, tw);
      break;
    default:
      break;
  }
}

// ---------------------------------------------------------------------------
// The same Stockham FFT with every size known at compile time: the
// transform length 2^LOGN, NFFT transforms, their strides, and the block
// shape.  Address arithmetic then folds into constants; where a stride is a
// multiple of 16 the padding of a whole run of 16 accesses is computed once
// (padi(a + 16 m) = padi(a) + 17 m).
// ---------------------------------------------------------------------------
template <int S> __device__ __forceinline__ int pad_step(int a, int r) {
  if constexpr (S % 16 == 0) return a + r * (S + S / 16);
  else return a + r * S;  // unused: callers branch on S % 16 first
}

template <typename R, int RAD, int LOGN, int LOGNS, int NFFT, int FSTRIDE, int ESTRIDE, int T,
          bool F_FAST>
__device__ __forceinline__ void stockham_pass_ct(typename RT<R>::C* buf, const typename RT<R>::C* tw) {
  using C = typename RT<R>::C;
  constexpr int LOGRAD = RAD == 2 ? 1 : RAD == 4 ? 2 : RAD == 8 ? 3 : 4;
  constexpr int LOGNB = LOGN - LOGRAD;
  constexpr int NB = 1 << LOGNB;
  constexpr int TOTAL = NFFT << LOGNB;
  constexpr int NS = 1 << LOGNS;
  constexpr int TWSHIFT = LOGN - LOGRAD - LOGNS;
  constexpr int MAXI = (TOTAL + T - 1) / T;
  constexpr int RSTR = NB * ESTRIDE;   // read stride between the RAD inputs
  constexpr int WSTR = NS * ESTRIDE;   // write stride between the RAD outputs
  C v[MAXI][RAD];
  int woff[MAXI];
#pragma unroll
  for (int it = 0; it < MAXI; ++it) {
    const int item = threadIdx.x + it * T;
    if (TOTAL % T == 0 || item < TOTAL) {
      int f, j;
      if (F_FAST) {
        f = item % NFFT;
        j = item / NFFT;
      } else {
        f = item >> LOGNB;
        j = item & (NB - 1);
      }
      const int k = j & (NS - 1);
      const int a = f * FSTRIDE + j * ESTRIDE;
      if constexpr (RSTR % 16 == 0) {
        const int pa = padi(a);
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[it][r] = buf[pad_step<RSTR>(pa, r)];
      } else {
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[it][r] = buf[padi(a + r * RSTR)];
      }
      if constexpr (LOGNS > 0) {
#pragma unroll
        for (int r = 1; r < RAD; ++r) v[it][r] = cmul(v[it][r], tw[(r * k) << TWSHIFT]);
      }
      dft_reg<RAD>(v[it]);
      woff[it] = f * FSTRIDE + (((j - k) << LOGRAD) + k) * ESTRIDE;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < MAXI; ++it) {
    const int item = threadIdx.x + it * T;
    if (TOTAL % T == 0 || item < TOTAL) {
      if constexpr (WSTR % 16 == 0) {
        const int pw = padi(woff[it]);
#pragma unroll
        for (int r = 0; r < RAD; ++r) buf[pad_step<WSTR>(pw, r)] = v[it][out_pos<RAD>(r)];
      } else {
#pragma unroll
        for (int r = 0; r < RAD; ++r) buf[padi(woff[it] + r * WSTR)] = v[it][out_pos<RAD>(r)];
      }
    }
  }
  __syncthreads();
}

template <typename R, int LOGN, int LOGNS, int NFFT, int FSTRIDE, int ESTRIDE, int T, bool F_FAST>
__device__ __forceinline__ void block_fft_ct_from(typename RT<R>::C* buf, const typename RT<R>::C* tw) {
  constexpr int REM = LOGN - LOGNS;
  if constexpr (REM >= 4) {
    stockham_pass_ct<R, 16, LOGN, LOGNS, NFFT, FSTRIDE, ESTRIDE, T, F_FAST>(buf, tw);
    block_fft_ct_from<R, LOGN, LOGNS + 4, NFFT, FSTRIDE, ESTRIDE, T, F_FAST>(buf, tw);
  } else if constexpr (REM == 3) {
    stockham_pass_ct<R, 8, LOGN, LOGNS, NFFT, FSTRIDE, ESTRIDE, T, F_FAST>(buf, tw);
  } else if constexpr (REM == 2) {
    stockham_pass_ct<R, 4, LOGN, LOGNS, NFFT, FSTRIDE, ESTRIDE, T, F_FAST>(buf, tw);
  } else if constexpr (REM == 1) {
    stockham_pass_ct<R, 2, LOGN, LOGNS, NFFT, FSTRIDE, ESTRIDE, T, F_FAST>(buf, tw);
  }
}

template <typename R, int LOGN, int NFFT, int FSTRIDE, int ESTRIDE, int T, bool F_FAST>
__device__ __forceinline__ void block_fft_ct(typename RT<R>::C* buf, const typename RT<R>::C* tw) {
  block_fft_ct_from<R, LOGN, 0, NFFT, FSTRIDE, ESTRIDE, T, F_FAST>(buf, tw);
}

// ---------------------------------------------------------------------------
// Mixed-radix Stockham FFT for any length n (the general-size path).
//
// The radices r_0, r_1, ... (product n) are applied in order.  The pass
// with radix RAD and span Ns = r_0 ... r_(p-1) maps x to y with
//   butterfly j < n / RAD,  k = j mod Ns:
//   v_r = x[j + r n / RAD] W_n^(r k n / (Ns RAD)),  V = DFT_RAD(v),
//   y[(j - k) RAD + k + r Ns] = V_r,
// which leaves the spectrum in natural order after the last pass (the same
// self-sorting scheme as the power-of-two passes above, with any radix).
// x and y are different buffers.  tw[t] = exp(-2 pi i t / n); the twiddle
// index r k n / (Ns RAD) stays below n.
// ---------------------------------------------------------------------------

// RAD-point forward DFT by its definition, natural order in and out, with
// W_RAD^q = tw[q * tstep] (tstep = n / RAD).
template <int RAD, typename C>
__device__ __forceinline__ void dft_def(C* v, const C* tw, int tstep) {
  C out[RAD];
#pragma unroll
  for (int r = 0; r < RAD; ++r) {
    out[r] = v[0];
#pragma unroll
    for (int m = 1; m < RAD; ++m) out[r] = cadd(out[r], cmul(v[m], tw[((r * m) % RAD) * tstep]));
  }
#pragma unroll
  for (int r = 0; r < RAD; ++r) v[r] = out[r];
}

// One butterfly of a pass with a radix known at compile time (2, 4, 8, 16
// by the register DFTs, 3, 5, 7 by definition).
template <int RAD, typename C>
__device__ __forceinline__ void any_butterfly(const C* x, C* y, int j, int n, int Ns, const C* tw) {
  const int nb = n / RAD, k = j % Ns, ts = n / (Ns * RAD);
  C v[RAD];
#pragma unroll
  for (int r = 0; r < RAD; ++r) v[r] = x[j + r * nb];
  if (k) {
#pragma unroll
    for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], tw[r * k * ts]);
  }
  const int o = (j - k) * RAD + k;
  if constexpr (RAD == 2 || RAD == 4 || RAD == 8 || RAD == 16) {
    dft_reg<RAD>(v);
#pragma unroll
    for (int r = 0; r < RAD; ++r) y[o + r * Ns] = v[out_pos<RAD>(r)];
  } else {
    dft_def<RAD>(v, tw, nb);
#pragma unroll
    for (int r = 0; r < RAD; ++r) y[o + r * Ns] = v[r];
  }
}

// Output r of one butterfly for any other radix (a prime above 7), summed
// straight from x (O(RAD) work; a pass spreads its outputs over threads);
// the combined exponent of the pass twiddle and W_RAD^(r m) is reduced
// modulo n.
template <typename C>
__device__ __forceinline__ void any_output_prime(const C* x, C* y, int j, int r, int rad, int n,
                                                 int Ns, const C* tw) {
  const int nb = n / rad, k = j % Ns, ts = n / (Ns * rad);
  const int o = (j - k) * rad + k;
  C acc = x[j];
  for (int m = 1; m < rad; ++m) {
    const long long e = (long long)m * k * ts + (long long)((r * m) % rad) * nb;
    acc = cadd(acc, cmul(x[j + m * nb], tw[(int)(e % n)]));
  }
  y[o + r * Ns] = acc;
}

}  // namespace rsx
