// CUDA kernels of the GB300 P-RSoXS path (sm_103a).
//
// Per energy and e-field angle the hot path (FP32, nx and ny 1024 or 512) runs:
//   k_pol_fft4s_tma  Eqs. (ncorr), (nrot), (polarization) and p <- U^T p for
//                    whole x-rows, fed by bulk copies, then the rows' x-FFT;
//                    p is never written before its first FFT pass.
//   k_yz_tma         the y-FFT of each z-slice (tiles by 2-D tensor copies)
//   (k_yz512_tma)    fused with the z-transform at the two q_z bins every
//                    pixel needs (Eq. (Ewald)), accumulated across z.
//   k_ewald_bins     Eqs. (3Dscatter) and (Ewald) from those bins; no 3-D X
//                    array exists.
//   k_rotate_acc     detector rotation about q = 0 and accumulation (Sec. 4).
// The general-size kernels (Stockham FFTs in shared memory: k_pol_fftx,
// k_col_fft, k_ewald_pruned / k_ewald_tma), the four-step variants with
// plain loads (FP64), Algorithm 2's N_t kernels and the linearity path's
// kernels follow.  None of the path is a dense contraction: the x pass is
// HBM-bound, the fused y+z pass bound by instruction issue.
#include <cuda.h>  // CUtensorMap (the type only; the library does not link libcuda)
#include <math.h>
#include <string.h>

#include <type_traits>

#include "rsx_device.cuh"
#include "rsx_kernels.h"

namespace rsx {

constexpr double kFourPi = 12.566370614359172953850573533118;

__host__ __device__ constexpr int ilog2_ct(int n) { return n <= 1 ? 0 : 1 + ilog2_ct(n >> 1); }

// ------------------------------------------------------------ polarisation
// Accumulated per voxel over components j, with a = v (1 + tau'_j),
// tau'_j = tau_j + s dperp_j, b = v s dpar_j and d_j the director:
//   (a^2 - 1)      = (v^2 - 1) + v^2 tau' (2 + tau')
//   (2ab + b^2)    = b (2 v (1 + tau') + b)
//   p = sum_j [(a_j^2 - 1) e + (2 a_j b_j + b_j^2)(d_j . e) d_j] / (4 pi)
// This is N_rot = a I + b d d^T squared (d d^T idempotent) for the uniaxial
// tensor of Eq. (uniaxialRefrativeIndex) rotated by R = B C D (Eq. nrot).
// The sum of (v^2 - 1) is kept apart as sum v^2 so that, together with the
// constant -(c-1), the large vacuum-like part never mixes with the small
// optical contrast in FP32.
template <typename R> struct PolAcc {
  R aw;         // sum_j v_j^2
  R as[2];      // sum_j v_j^2 tau'_j (2 + tau'_j)
  R b[3][2];    // sum_j (2ab + b^2)(d . e) d
};

template <typename R>
__device__ __forceinline__ void pol_zero(PolAcc<R>& a) {
  a.aw = 0;
  a.as[0] = a.as[1] = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) a.b[k][0] = a.b[k][1] = 0;
}

// FP32: the SFU approximation, which is accurate (absolute error ~1e-6) only
// near [-pi, pi].  The Euler angles of Sec. 3.1 are not restricted, so x is
// first reduced to r = x - n 2 pi, n = rint(x / 2 pi), by Cody and Waite's
// method with a two-part constant: hi = float(2 pi), lo = float(2 pi - hi),
// each product subtracted in one fused multiply-add.  For |x| up to ~1e4
// the reduced angle is off by less than one ulp of pi, far below the FP32
// contrast tolerance.  FP64 keeps the library call, which reduces any range.
__device__ __forceinline__ float reduce_2pi(float x) {
  constexpr double two_pi = 6.283185307179586476925286766559;
  constexpr float hi = (float)two_pi;
  constexpr float lo = (float)(two_pi - (double)hi);
  const float n = rintf(x * (float)(1.0 / two_pi));
  return fmaf(-n, lo, fmaf(-n, hi, x));
}
__device__ __forceinline__ void sincos_r(float x, float* s, float* c) {
  __sincosf(reduce_2pi(x), s, c);
}
__device__ __forceinline__ void sincos_r(double x, double* s, double* c) { sincos(x, s, c); }

// The same with the director d = (dx, dy, dz) of component j given.
template <typename R>
__device__ __forceinline__ void pol_add_d(PolAcc<R>& acc, R v, R s, R dx, R dy, R dz,
                                          const PolParams<R>& pp, int j) {
  const R v2 = v * v, v2s = v2 * s, v2s2 = v2s * s;
  acc.aw += v2;
  acc.as[0] += v2 * pp.q[j][0][0] + v2s * pp.q[j][1][0] + v2s2 * pp.q[j][2][0];
  acc.as[1] += v2 * pp.q[j][0][1] + v2s * pp.q[j][1][1] + v2s2 * pp.q[j][2][1];
  const R gr = v2s * pp.q[j][3][0] + v2s2 * pp.q[j][4][0];
  const R gi = v2s * pp.q[j][3][1] + v2s2 * pp.q[j][4][1];
  const R de = dx * pp.ce + dy * pp.se;
  const R hr = gr * de, hi = gi * de;
  acc.b[0][0] += hr * dx; acc.b[0][1] += hi * dx;
  acc.b[1][0] += hr * dy; acc.b[1][1] += hi * dy;
  acc.b[2][0] += hr * dz; acc.b[2][1] += hi * dz;
}

template <typename R>
__device__ __forceinline__ void pol_add(PolAcc<R>& acc, R v, R s, R phi, R theta,
                                        const PolParams<R>& pp, int j) {
  const R v2 = v * v, v2s = v2 * s, v2s2 = v2s * s;
  acc.aw += v2;
  // v^2 tau' (2 + tau')
  acc.as[0] += v2 * pp.q[j][0][0] + v2s * pp.q[j][1][0] + v2s2 * pp.q[j][2][0];
  acc.as[1] += v2 * pp.q[j][0][1] + v2s * pp.q[j][1][1] + v2s2 * pp.q[j][2][1];
  // g = b (2 a + b) with a = v (1 + tau'), b = v s dpar
  const R gr = v2s * pp.q[j][3][0] + v2s2 * pp.q[j][4][0];
  const R gi = v2s * pp.q[j][3][1] + v2s2 * pp.q[j][4][1];
  R sp, cp, st, ct;
  sincos_r(phi, &sp, &cp);
  sincos_r(theta, &st, &ct);
  const R dx = cp * st, dy = sp * st, dz = ct;
  const R de = dx * pp.ce + dy * pp.se;
  const R hr = gr * de, hi = gi * de;
  acc.b[0][0] += hr * dx; acc.b[0][1] += hi * dx;
  acc.b[1][0] += hr * dy; acc.b[1][1] += hi * dy;
  acc.b[2][0] += hr * dz; acc.b[2][1] += hi * dz;
}

// p (minus the reference constant unless add_ref) in the frame of pp.literal.
template <typename R>
__device__ __forceinline__ void pol_final(const PolAcc<R>& acc, const PolParams<R>& pp,
                                          typename RT<R>::C out[3]) {
  const R inv = R(1.0 / kFourPi);
  R ar = (acc.aw - R(1)) + acc.as[0];
  if (pp.add_ref) ar -= R(pp.c - 1);
  const R ai = acc.as[1];
  const R ce = pp.ce, se = pp.se;
  R p0r, p0i, p1r, p1i;
  if (pp.literal) {
    p0r = ar + ce * acc.b[0][0] + se * acc.b[1][0];
    p0i = ai + ce * acc.b[0][1] + se * acc.b[1][1];
    p1r = -se * acc.b[0][0] + ce * acc.b[1][0];
    p1i = -se * acc.b[0][1] + ce * acc.b[1][1];
  } else {
    p0r = ar * ce + acc.b[0][0];
    p0i = ai * ce + acc.b[0][1];
    p1r = ar * se + acc.b[1][0];
    p1i = ai * se + acc.b[1][1];
  }
  out[0] = RT<R>::mk(p0r * inv, p0i * inv);
  out[1] = RT<R>::mk(p1r * inv, p1i * inv);
  out[2] = RT<R>::mk(acc.b[2][0] * inv, acc.b[2][1] * inv);
}

// Loads of data read once per pass (the morphology, N_t): streaming hint, so
// that they do not push the x-transformed slices out of L2 before the y pass
// reads them back.
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ double4_32a ld_stream(const double4_32a* p) { return *p; }
__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }

template <typename R>
__device__ __forceinline__ void load_m(const typename RT<R>::V4* M, size_t i, R& v, R& s, R& ph,
                                       R& th) {
  const typename RT<R>::V4 m = M[i];
  v = m.x; s = m.y; ph = m.z; th = m.w;
}

// One CTA: ROWS = EC / nx consecutive x-rows (row = z * ny + y) of all three
// components of p.  Polarisation is computed component-outer, the loads of
// component j + 1 issued before the arithmetic of component j, so that every
// thread keeps 2 SLOTS independent 16/32-byte loads in flight; then the
// 3*ROWS rows are transformed along x in shared memory and written once.
// LOGNX >= 0 fixes nx = 2^LOGNX at compile time (the FFT's index arithmetic
// then folds into constants); LOGNX < 0 takes lognx at run time.
// FROM_NT: the source is Algorithm 2's N_t (five complex entries per voxel,
// nt[5][N] = xx, xy, yy, xz, yz, with the same constant removed from the
// diagonal) instead of the morphology, and p = N_t . e.
template <typename R, int T, int EC, bool DO_FFT, int LOGNX, bool FROM_NT>
__global__ void __launch_bounds__(T, (sizeof(R) == 4 && EC <= 1024) ? 3 : 1) k_pol_fftx(const typename RT<R>::V4* __restrict__ M,
                                                long long N, int lognx_rt, long long row_begin,
                                                long long row_end, PolParams<R> pp,
                                                typename RT<R>::C* __restrict__ p,
                                                const typename RT<R>::C* __restrict__ twx,
                                                int tw_in_smem,
                                                const typename RT<R>::C* __restrict__ nt,
                                                const R* __restrict__ dir) {
  using C = typename RT<R>::C;
  using V4 = typename RT<R>::V4;
  constexpr int SLOTS = EC / T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [3][ROWS][nx], padded
  C* tws = buf + padded(3 * EC);
  const int lognx = LOGNX >= 0 ? LOGNX : lognx_rt;
  const int nx = 1 << lognx;
  const int ROWS = EC >> lognx;
  const long long row0 = row_begin + (long long)blockIdx.x * ROWS;
  const long long rl = row_end - row0;
  const int rows_here = rl < ROWS ? (int)rl : ROWS;
  const int nel = rows_here << lognx;
  const size_t vox0 = (size_t)row0 << lognx;

  if (DO_FFT && tw_in_smem)
    for (int i = threadIdx.x; i < nx; i += T) tws[i] = twx[i];

  if constexpr (FROM_NT) {
    const R inv_ref = pp.add_ref ? R(-(pp.c - 1) / kFourPi) : R(0);
#pragma unroll
    for (int sl = 0; sl < SLOTS; ++sl) {
      const int e = threadIdx.x + sl * T;
      if (e < nel) {
        const size_t i = vox0 + e;
        C t[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) t[q] = ld_stream(nt + q * (size_t)N + i);
        const R ce = pp.ce, se = pp.se;
        // p = N_t . e with e = (ce, se, 0): columns x and y of N_t
        C px = RT<R>::mk(t[0].x * ce + t[1].x * se + inv_ref * ce, t[0].y * ce + t[1].y * se);
        C py = RT<R>::mk(t[1].x * ce + t[2].x * se + inv_ref * se, t[1].y * ce + t[2].y * se);
        const C pz = RT<R>::mk(t[3].x * ce + t[4].x * se, t[3].y * ce + t[4].y * se);
        C out[3];
        if (pp.literal) {
          out[0] = RT<R>::mk(ce * px.x + se * py.x, ce * px.y + se * py.y);
          out[1] = RT<R>::mk(-se * px.x + ce * py.x, -se * px.y + ce * py.y);
        } else {
          out[0] = px;
          out[1] = py;
        }
        out[2] = pz;
        if (DO_FFT) {
          buf[padi(e)] = out[0];
          buf[padi(EC + e)] = out[1];
          buf[padi(2 * EC + e)] = out[2];
        } else {
          p[i] = out[0];
          p[(size_t)N + i] = out[1];
          p[2 * (size_t)N + i] = out[2];
        }
      }
    }
  } else {
  PolAcc<R> acc[SLOTS];
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) pol_zero(acc[sl]);
  V4 cur[SLOTS], nxt[SLOTS];
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int e = threadIdx.x + sl * T;
    if (e < nel) cur[sl] = ld_stream(M + vox0 + e);
  }
  for (int j = 0; j < pp.c; ++j) {
    if (j + 1 < pp.c) {
      const V4* Mj = M + (size_t)(j + 1) * N + vox0;
#pragma unroll
      for (int sl = 0; sl < SLOTS; ++sl) {
        const int e = threadIdx.x + sl * T;
        if (e < nel) nxt[sl] = ld_stream(Mj + e);
      }
    }
    if (dir) {  // the cached director of component j ([c][3][N])
      const R* dj = dir + (size_t)j * 3 * N + vox0;
#pragma unroll
      for (int sl = 0; sl < SLOTS; ++sl) {
        const int e = threadIdx.x + sl * T;
        if (e < nel)
          pol_add_d(acc[sl], (R)cur[sl].x, (R)cur[sl].y, dj[e], dj[N + e], dj[2 * N + e], pp, j);
      }
    } else {
#pragma unroll
      for (int sl = 0; sl < SLOTS; ++sl) {
        const int e = threadIdx.x + sl * T;
        if (e < nel)
          pol_add(acc[sl], (R)cur[sl].x, (R)cur[sl].y, (R)cur[sl].z, (R)cur[sl].w, pp, j);
      }
    }
#pragma unroll
    for (int sl = 0; sl < SLOTS; ++sl) cur[sl] = nxt[sl];
  }
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int e = threadIdx.x + sl * T;
    if (e < nel) {
      C out[3];
      pol_final(acc[sl], pp, out);
      if (DO_FFT) {
        buf[padi(e)] = out[0];
        buf[padi(EC + e)] = out[1];
        buf[padi(2 * EC + e)] = out[2];
      } else {
        p[vox0 + e] = out[0];
        p[(size_t)N + vox0 + e] = out[1];
        p[2 * (size_t)N + vox0 + e] = out[2];
      }
    }
  }
  }
  if (!DO_FFT) return;
  __syncthreads();
  const C* tw = tw_in_smem ? tws : twx;
  if constexpr (LOGNX >= 0)
    block_fft_ct<R, LOGNX, 3 * (EC >> LOGNX), (1 << LOGNX), 1, T, false>(buf, tw);
  else
    block_fft<R, 3 * EC, T, false>(buf, lognx, 3 * ROWS, -1, nx, 1, tw);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    for (int e = threadIdx.x; e < nel; e += T) p[(size_t)k * N + vox0 + e] = buf[padi(k * EC + e)];
}

// ------------------------------------------------- four-step 1024-point FFTs
// N = 1024 = 32 x 32: with n = n1 + 32 n2 and k = k2 + 32 k1,
//   X[k2 + 32 k1] = sum_n1 W32^(n1 k1) W1024^(n1 k2) sum_n2 x[n1 + 32 n2] W32^(n2 k2).
// A thread owning n1 holds the 32 samples n2 in registers (32-point DFT),
// multiplies by W1024^(n1 k2) (table tw4[k2 * 32 + n1]), and after one
// transpose through shared memory a thread owning k2 does the second
// 32-point DFT and holds X[k2 + 32 k1] for k1 = 0..31.  One shared-memory
// round trip instead of three Stockham passes.

// x pass: polarisation of one row into shared memory by four warps (eight
// voxels per thread, component loads double-buffered), then warps 0..2 each
// transform one field with warp-level synchronisation only, writing the
// spectrum straight from registers (coalesced over k2).
template <typename R, bool FROM_NT>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 4 : 1) k_pol_fft4s(const typename RT<R>::V4* __restrict__ M,
                                                      long long N, long long nrows, PolParams<R> pp,
                                                      typename RT<R>::C* __restrict__ p,
                                                      const typename RT<R>::C* __restrict__ tw4_g,
                                                      const typename RT<R>::C* __restrict__ nt,
                                                      const R* __restrict__ dir) {
  using C = typename RT<R>::C;
  using V4 = typename RT<R>::V4;
  constexpr int T = 128, NX = 1024, SLOTS = NX / T, FS = 32 * 33;  // field stride in smem
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);  // [3][32 * 33]
  C* tw4 = P + 3 * FS;                     // [32][32]
  const long long row = blockIdx.x;
  if (row >= nrows) return;
  const size_t vox0 = (size_t)row * NX;
  for (int i = threadIdx.x; i < NX; i += T) tw4[i] = tw4_g[i];

  if constexpr (FROM_NT) {
    const R inv_ref = pp.add_ref ? R(-(pp.c - 1) / kFourPi) : R(0);
#pragma unroll
    for (int sl = 0; sl < SLOTS; ++sl) {
      const int e = threadIdx.x + sl * T;
      const size_t i = vox0 + e;
      C t[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) t[q] = ld_stream(nt + q * (size_t)N + i);
      const R ce = pp.ce, se = pp.se;
      const C px = RT<R>::mk(t[0].x * ce + t[1].x * se + inv_ref * ce, t[0].y * ce + t[1].y * se);
      const C py = RT<R>::mk(t[1].x * ce + t[2].x * se + inv_ref * se, t[1].y * ce + t[2].y * se);
      const C pz = RT<R>::mk(t[3].x * ce + t[4].x * se, t[3].y * ce + t[4].y * se);
      if (pp.literal) {
        P[e] = RT<R>::mk(ce * px.x + se * py.x, ce * px.y + se * py.y);
        P[FS + e] = RT<R>::mk(-se * px.x + ce * py.x, -se * px.y + ce * py.y);
      } else {
        P[e] = px;
        P[FS + e] = py;
      }
      P[2 * FS + e] = pz;
    }
  } else {
    // component-outer: all eight loads of a component issued, then used
    PolAcc<R> acc[SLOTS];
#pragma unroll
    for (int sl = 0; sl < SLOTS; ++sl) pol_zero(acc[sl]);
    for (int j = 0; j < pp.c; ++j) {
      const V4* Mj = M + (size_t)j * N + vox0;
      V4 cur[SLOTS];
#pragma unroll
      for (int sl = 0; sl < SLOTS; ++sl) cur[sl] = ld_stream(Mj + threadIdx.x + sl * T);
      if (dir) {  // the cached director of component j ([c][3][N])
        const R* dj = dir + (size_t)j * 3 * N + vox0 + threadIdx.x;
#pragma unroll
        for (int sl = 0; sl < SLOTS; ++sl)
          pol_add_d(acc[sl], (R)cur[sl].x, (R)cur[sl].y, dj[sl * T], dj[N + sl * T],
                    dj[2 * N + sl * T], pp, j);
      } else {
#pragma unroll
        for (int sl = 0; sl < SLOTS; ++sl)
          pol_add(acc[sl], (R)cur[sl].x, (R)cur[sl].y, (R)cur[sl].z, (R)cur[sl].w, pp, j);
      }
    }
#pragma unroll
    for (int sl = 0; sl < SLOTS; ++sl) {
      const int e = threadIdx.x + sl * T;
      C out[3];
      pol_final(acc[sl], pp, out);
      P[e] = out[0];
      P[FS + e] = out[1];
      P[2 * FS + e] = out[2];
    }
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w >= 3) return;
  C* F = P + w * FS;
  C v[32];
#pragma unroll
  for (int n2 = 0; n2 < 32; ++n2) v[n2] = F[lane + 32 * n2];
  dft32(v);
#pragma unroll
  for (int k2 = 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], tw4[k2 * 32 + lane]);
  __syncwarp();
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) F[k2 * 33 + lane] = v[k2];
  __syncwarp();
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) v[n1] = F[lane * 33 + n1];
  dft32(v);
  C* out = p + (size_t)w * N + vox0 + lane;
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) out[32 * k1] = v[k1];
}

// One warp's x-FFT of one field of a row held in shared memory (F, padded
// as [NX / 32][33]) and its store to out_row[0 .. NX).  release() runs once
// the warp has read F for the last time, before the second DFT and the
// stores, so the row buffer can be refilled while they run.
//  NX = 1024 = 32 x 32: as k_pol_fft4s.
//  NX = 512 = 32 x 16 with n = n1 + 32 n2, k = k2 + 16 k1: lane n1 does the
//  16-point DFT over n2 and the twiddles W512^(n1 k2) (tw4: W512^j); after
//  the transpose, lanes k2 and k2 + 16 share the 32-point DFT over n1 (even
//  n1 on the lower lane, odd on the upper), which leaves k1 = k and
//  k1 = 16 + k on the two lanes.
// One warp's 1024-point four-step FFT of F (dense elements 0..1023, then
// transposed in place as [32][33]); output k goes to out[OS * k].
template <int OS, typename Release>
__device__ __forceinline__ void fft1024_warp(float2* F, const float2* tw4, float2* out, int lane,
                                             Release release) {
  using C = float2;
  C v[32];
#pragma unroll
  for (int n2 = 0; n2 < 32; ++n2) v[n2] = F[lane + 32 * n2];
  dft32(v);
#pragma unroll
  for (int k2 = 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], tw4[k2 * 32 + lane]);
  __syncwarp();
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) F[k2 * 33 + lane] = v[k2];
  __syncwarp();
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) v[n1] = F[lane * 33 + n1];
  __syncwarp();
  release();
  dft32(v);
  C* o = out + OS * lane;
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) o[OS * 32 * k1] = v[k1];
}

template <int NX, typename Release>
__device__ __forceinline__ void xfft_row(float2* F, const float2* tw4, float2* out_row, int lane,
                                         Release release) {
  using C = float2;
  C v[32];
  if constexpr (NX == 1024) {
    fft1024_warp<1>(F, tw4, out_row, lane, release);
  } else if constexpr (NX == 2048) {
    // decimation in frequency: X[2k] and X[2k + 1] are the 1024-point
    // transforms of a[n] = x[n] + x[n + 1024] and b[n] = (x[n] - x[n + 1024])
    // W2048^n; F holds x[0..1024) at 0.. and x[1024..2048) at 1056..,
    // tw4[1024 + n] = W2048^n
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      const int n = lane + 32 * j;
      const C a = F[n], b = F[1056 + n];
      F[n] = cadd(a, b);
      F[1056 + n] = cmul(csub(a, b), tw4[1024 + n]);
    }
    __syncwarp();
    fft1024_warp<2>(F, tw4, out_row, lane, [] {});
    fft1024_warp<2>(F + 1056, tw4, out_row + 1, lane, release);
  } else {
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) v[n2] = F[lane + 32 * n2];
    dft_reg<16>(v);
    C u[16];
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) u[k2] = cmul(v[out_pos<16>(k2)], tw4[lane * k2]);
    __syncwarp();
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) F[k2 * 33 + lane] = u[k2];
    __syncwarp();
    const int k2 = lane & 15, h = lane >> 4;
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = F[k2 * 33 + 2 * m + h];
    __syncwarp();
    release();
    dft32_pair(v, u, h);
    C* out = out_row + k2 + 256 * h;
#pragma unroll
    for (int k = 0; k < 16; ++k) out[16 * k] = u[k];
  }
}

// x pass (FP32, nx = NX = 1024 or 512) as a warp-specialised bulk-copy
// pipeline, for Algorithm 1 (NT = false: the morphology, c slices of 16 NX
// bytes per row) or Algorithm 2 (NT = true: the five stored entries of N_t,
// 8 NX bytes each).
// Three roles per block:
//  * a producer lane streams (row, component or entry) slices into a ring
//    of S shared-memory stages (full/empty mbarrier pairs), up to S slices
//    ahead;
//  * PW polarisation warps accumulate NX / (32 PW) voxels per thread from
//    each stage (Algorithm 1: pol_add per component; Algorithm 2: p = N_t e
//    entry by entry), release it per warp, and write the row's three fields
//    into one of NP row buffers;
//  * FG groups of three transform warps (group g takes the rows r with
//    r mod FG = g) run a four-step FFT on a filled buffer (32 x 32 as in
//    k_pol_fft4s, or 32 x 16 for 512 points) and store the spectrum.
// Row buffers pass between the roles on named barriers (full: 1 + i, empty:
// 1 + NP + i), so polarisation of the next rows overlaps the transforms.
// CTAs are persistent and walk rows with a grid stride.  Every mbarrier wait
// is bounded; a timeout sets *err and the block's abort flag, after which the
// roles skip their work but still complete the barrier protocol (which has
// no unbounded wait left), the producer waits (bounded) for its copies in
// flight, and the block exits.
template <int S, int NP, int PW, int FG, bool NT, int NX>
__global__ void __launch_bounds__(32 * (PW + 3 * FG + 1)) k_pol_fft4s_tma(
    const void* __restrict__ src, long long N, long long nrows, PolParams<float> pp,
    float2* __restrict__ p, const float2* __restrict__ tw4_g, int* __restrict__ err,
    unsigned poll) {
  using C = float2;
  using SrcT = typename std::conditional<NT, float2, float4>::type;
  static_assert(NX == 1024 || NX == 512, "row length");
  // row buffers: the 1024-point transform's 32 x 33 transpose; 512 points
  // transpose 16 x 33 (tw4_g: W1024^(ab) as [32][32], or W512^j for 512)
  constexpr int TP = 32 * PW, SL = NX / TP, FS = (NX / 32) * 33, NB = TP + 96;
  static_assert(NX % TP == 0 && 1 + 2 * NP <= 15 && NP % FG == 0, "layout");
  constexpr unsigned kPoll = 1u << 22, kStageBytes = NX * sizeof(SrcT);
  extern __shared__ __align__(128) unsigned char smem_a128[];
  SrcT* stage = reinterpret_cast<SrcT*>(smem_a128);        // [S][NX]
  C* P = reinterpret_cast<C*>(stage + S * NX);             // [NP][3][FS]
  C* tw4 = P + NP * 3 * FS;                                 // [32][32]
  unsigned long long* full = reinterpret_cast<unsigned long long*>(tw4 + 1024);
  unsigned long long* empty = full + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (t == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], PW);
    }
    *abort_flag = 0;
    fence_proxy_async();
  }
  for (int i = t; i < (NX == 1024 ? 1024 : 512); i += blockDim.x) tw4[i] = tw4_g[i];
  __syncthreads();
  const long long nmine =
      blockIdx.x < nrows ? (nrows - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (w == PW + 3 * FG) {  // producer warp, one lane
    if (lane != 0) return;
    // stage g = rr * c + j goes to slot g mod S; its k-th reuse (k = g / S)
    // waits for the k-1-th release.  32-bit counters (g < 2^31).
    const int per_row = NT ? 5 : pp.c;
    const int G = (int)nmine * per_row;
    const SrcT* M = reinterpret_cast<const SrcT*>(src);
    int g = 0, slot = 0, k = 0, j = 0;
    long long row = blockIdx.x;
    for (; g < G; ++g) {
      if (k > 0 && !mbar_wait_bounded(&empty[slot], (unsigned)((k - 1) & 1), poll)) {
        atomicOr(err, 1);
        *abort_flag = 1;
        break;
      }
      mbar_expect_tx(&full[slot], kStageBytes);
      bulk_g2s(stage + slot * NX, M + (size_t)j * N + (size_t)row * NX, kStageBytes, &full[slot]);
      if (++slot == S) slot = 0, ++k;
      if (++j == per_row) j = 0, row += gridDim.x;
    }
    // nothing may be in flight when the block exits
    for (int d = g - 1; d >= 0 && d >= g - S; --d)
      mbar_wait_bounded(&full[d % S], (unsigned)((d / S) & 1), kPoll);
    return;
  }

  if (w < PW) {  // polarisation warps
    bool failed = false;
    const int per_row = NT ? 5 : pp.c;
    int slot = 0, ph = 0;  // stage rr * per_row + j: its slot and the parity of its use
    for (int rr = 0; rr < (int)nmine; ++rr) {
      PolAcc<float> acc[SL];  // Algorithm 1
      C pe[SL][3];            // Algorithm 2: p = N_t e, before the frame rotation
#pragma unroll
      for (int sl = 0; sl < SL; ++sl) {
        if constexpr (NT) {
          pe[sl][0] = pe[sl][1] = pe[sl][2] = make_float2(0.f, 0.f);
        } else {
          pol_zero(acc[sl]);
        }
      }
      for (int j = 0; j < per_row; ++j) {
        const int cs = slot, cph = ph;
        if (++slot == S) slot = 0, ph ^= 1;
        failed = failed || __any_sync(0xffffffffu, *abort_flag != 0);
        if (failed) break;
        // warp-uniform: a lane that gave up makes its whole warp give up
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[cs], (unsigned)cph, poll))) {
          failed = true;
          atomicOr(err, 1);
          *abort_flag = 1;
          break;
        }
        const SrcT* st = stage + cs * NX;
        SrcT cur[SL];
#pragma unroll
        for (int sl = 0; sl < SL; ++sl) cur[sl] = st[t + sl * TP];
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[cs]);
        if constexpr (NT) {
          // entries xx, xy, yy, xz, yz of the symmetric N_t times e = (ce, se, 0):
          // px = xx ce + xy se, py = xy ce + yy se, pz = xz ce + yz se
          auto madd = [&](int f, float w) {
#pragma unroll
            for (int sl = 0; sl < SL; ++sl) {
              pe[sl][f].x += cur[sl].x * w;
              pe[sl][f].y += cur[sl].y * w;
            }
          };
          if (j == 0) {
            madd(0, pp.ce);
          } else if (j == 1) {
            madd(0, pp.se);
            madd(1, pp.ce);
          } else if (j == 2) {
            madd(1, pp.se);
          } else if (j == 3) {
            madd(2, pp.ce);
          } else {
            madd(2, pp.se);
          }
        } else {
#pragma unroll
          for (int sl = 0; sl < SL; ++sl)
            pol_add(acc[sl], cur[sl].x, cur[sl].y, cur[sl].z, cur[sl].w, pp, j);
        }
      }
      const int i = rr % NP;
      if (rr >= NP) named_bar_sync(1 + NP + i, NB);  // transforms of row rr - NP done
      if (!failed) {
        C* Pi = P + i * 3 * FS;
#pragma unroll
        for (int sl = 0; sl < SL; ++sl) {
          const int e = t + sl * TP;
          C out[3];
          if constexpr (NT) {
            // the reference constant returns as -(c-1)/(4 pi) e when add_ref
            const float inv_ref = pp.add_ref ? -(pp.c - 1) / (float)kFourPi : 0.f;
            const C px = make_float2(pe[sl][0].x + inv_ref * pp.ce, pe[sl][0].y);
            const C py = make_float2(pe[sl][1].x + inv_ref * pp.se, pe[sl][1].y);
            if (pp.literal) {
              out[0] = make_float2(pp.ce * px.x + pp.se * py.x, pp.ce * px.y + pp.se * py.y);
              out[1] = make_float2(-pp.se * px.x + pp.ce * py.x, -pp.se * px.y + pp.ce * py.y);
            } else {
              out[0] = px;
              out[1] = py;
            }
            out[2] = pe[sl][2];
          } else {
            pol_final(acc[sl], pp, out);
          }
          Pi[e] = out[0];
          Pi[FS + e] = out[1];
          Pi[2 * FS + e] = out[2];
        }
      }
      named_bar_arrive(1 + i, NB);
    }
    return;
  }

  // transform warps: group fg, field f
  const int fg = (w - PW) / 3, f = (w - PW) % 3;
  for (int rr = fg; rr < (int)nmine; rr += FG) {
    const int i = rr % NP;
    named_bar_sync(1 + i, NB);
    if (*abort_flag == 0) {
      const long long row = blockIdx.x + rr * gridDim.x;
      xfft_row<NX>(P + i * 3 * FS + f * FS, tw4, p + (size_t)f * N + (size_t)row * NX, lane, [&] {
        if (rr + NP < nmine) named_bar_arrive(1 + NP + i, NB);
      });
    } else if (rr + NP < nmine) {
      named_bar_arrive(1 + NP + i, NB);
    }
  }
}

// ------------------------------------------- x pass for several angles
// The angle-independent part of Eq. (polarization) at one voxel, summed
// over components j with g_j = b_j (2 a_j + b_j) (a_j = v (1 + tau'_j),
// b_j = v s dpar_j) and the director d_j:
//   p(e) = [ ((sum_j v_j^2 - 1) + sum_j v_j^2 tau'_j (2 + tau'_j)) e + T e ] / (4 pi),
//   T = sum_j g_j d_j d_j^T  (complex symmetric),
// of which e = (cos a, sin a, 0) meets only the entries xx, xy, yy, xz, yz.
// Summing T instead of T e lets one read of the morphology serve several
// e-field angles; each angle's p is then formed exactly as Eq.
// (polarization) prescribes (the same products, summed in another order).
struct TAcc {
  float aw;        // sum_j v_j^2
  float as[2];     // sum_j v_j^2 tau'_j (2 + tau'_j)
  float t[5][2];   // T: xx, xy, yy, xz, yz
};

__device__ __forceinline__ void tacc_zero(TAcc& a) {
  a.aw = 0.f;
  a.as[0] = a.as[1] = 0.f;
#pragma unroll
  for (int q = 0; q < 5; ++q) a.t[q][0] = a.t[q][1] = 0.f;
}

__device__ __forceinline__ void tacc_add(TAcc& acc, float v, float s, float phi, float theta,
                                         const PolParams<float>& pp, int j) {
  const float v2 = v * v, v2s = v2 * s, v2s2 = v2s * s;
  acc.aw += v2;
  acc.as[0] += v2 * pp.q[j][0][0] + v2s * pp.q[j][1][0] + v2s2 * pp.q[j][2][0];
  acc.as[1] += v2 * pp.q[j][0][1] + v2s * pp.q[j][1][1] + v2s2 * pp.q[j][2][1];
  const float gr = v2s * pp.q[j][3][0] + v2s2 * pp.q[j][4][0];
  const float gi = v2s * pp.q[j][3][1] + v2s2 * pp.q[j][4][1];
  float sp, cp, st, ct;
  sincos_r(phi, &sp, &cp);
  sincos_r(theta, &st, &ct);
  const float dx = cp * st, dy = sp * st, dz = ct;
  const float hxr = gr * dx, hxi = gi * dx, hyr = gr * dy, hyi = gi * dy;
  acc.t[0][0] += hxr * dx; acc.t[0][1] += hxi * dx;
  acc.t[1][0] += hxr * dy; acc.t[1][1] += hxi * dy;
  acc.t[2][0] += hyr * dy; acc.t[2][1] += hyi * dy;
  acc.t[3][0] += hxr * dz; acc.t[3][1] += hxi * dz;
  acc.t[4][0] += hyr * dz; acc.t[4][1] += hyi * dz;
}

// p for e = (c, s, 0) = (cos a, sin a, 0) from the sums, already divided by
// 4 pi (ar + i ai = [(sum v^2 - 1) + sum v^2 tau'(2 + tau')] / (4 pi), the
// reference constant left out; t = T / (4 pi)), in the frame of `literal`:
// with b = T e,
//   literal (p <- U^T p):  p0 = ar + c b_x + s b_y = ar + c^2 Txx + 2cs Txy + s^2 Tyy
//                          p1 = -s b_x + c b_y    = cs (Tyy - Txx) + (c^2 - s^2) Txy
//   lab:                   p0 = c ar + b_x,  p1 = s ar + b_y,
//   both:                  p2 = b_z = c Txz + s Tyz.
__device__ __forceinline__ void p_from_tacc(float ar, float ai, const float (&t)[5][2], float c,
                                            float s, bool literal, float2 out[3]) {
  if (literal) {
    const float c2 = c * c, s2 = s * s, cs2 = 2.f * c * s, cs = c * s, d2 = c2 - s2;
    out[0] = make_float2(fmaf(s2, t[2][0], fmaf(cs2, t[1][0], fmaf(c2, t[0][0], ar))),
                         fmaf(s2, t[2][1], fmaf(cs2, t[1][1], fmaf(c2, t[0][1], ai))));
    out[1] = make_float2(fmaf(d2, t[1][0], cs * (t[2][0] - t[0][0])),
                         fmaf(d2, t[1][1], cs * (t[2][1] - t[0][1])));
  } else {
    out[0] = make_float2(fmaf(c, ar + t[0][0], s * t[1][0]), fmaf(c, ai + t[0][1], s * t[1][1]));
    out[1] = make_float2(fmaf(s, ar + t[2][0], c * t[1][0]), fmaf(s, ai + t[2][1], c * t[1][1]));
  }
  out[2] = make_float2(fmaf(c, t[3][0], s * t[4][0]), fmaf(c, t[3][1], s * t[4][1]));
}

// The Algorithm 1 x pass for up to KMAX e-field angles per read of the
// morphology (FP32, nx = NX = 1024 or 512): the roles and the bulk-copy
// ring of k_pol_fft4s_tma, but the polarisation warps accumulate the
// angle-independent sums (TAcc) of their voxels over the c component
// stages, then form p for each angle k < ang.n in turn and hand it to the
// transform warps through a ring of NPB row buffers; the transform groups
// write angle k's spectrum to p + k * pstride.  Row buffer u = rr * n + k
// (row rr of this block, angle k) is slot u mod NPB, passed on named
// barriers (full: 1 + slot, empty: 1 + NPB + slot); NPB a multiple of FG
// keeps each slot with one transform group.  Per voxel and angle this
// reads 16 c / n bytes of morphology instead of 16 c.  One persistent CTA
// per SM.  Waits are bounded as in k_pol_fft4s_tma.
// Roles of the 18 warps of the multi-angle x pass (8 polarisation, 9
// transform, 1 producer).  A block's warps are dealt to the SM's four
// schedulers by warp index mod 4, and the transform warps carry about twice
// the per-warp work of the others, so they are spread 2, 2, 3, 2 over the
// schedulers with the polarisation warps and the producer filling the rest:
// kind 0 = polarisation (index 0..7), 1 = transform (index 0..8, group
// index / 3, field index mod 3), 2 = producer.
// Warps 0-7 and 10 transform (indices 0-7, 8), 16 produces, the other eight
// polarise (8, 9, 11, 12, 13, 14, 15, 17 -> 0..7).  (P1: x pass 85.7 -> 84.6
// ms per energy; the 2048-point rows, whose transforms are longer, keep warp
// order: 3 % slower with this table.)
__device__ __forceinline__ void multi_role(int w, int& kind, int& idx) {
  if (w < 8 || w == 10) {
    kind = 1;
    idx = w < 8 ? w : 8;
  } else if (w == 16) {
    kind = 2;
    idx = 0;
  } else {
    kind = 0;
    idx = w - 8 - (w > 10) - (w > 16);
  }
}

template <int S, int NPB, int PW, int FG, int NX, int KMAX>
__global__ void __launch_bounds__(32 * (PW + 3 * FG + 1), 1) k_pol_fft4s_tma_multi(
    const float4* __restrict__ M, long long N, long long nrows, PolParams<float> pp,
    XAngles ang, float2* __restrict__ p, long long pstride, const float2* __restrict__ tw4_g,
    int* __restrict__ err, unsigned poll) {
  using C = float2;
  static_assert(NX == 1024 || NX == 512 || NX == 2048, "row length");
  static_assert(KMAX <= kMaxXAngles, "angle set");
  // a stage is one component of a row segment of SV voxels; 2048-point rows
  // come in H = 2 segments, whose fields sit at 0 and 1056 of a row buffer
  constexpr int SV = NX > 1024 ? 1024 : NX, H = NX / SV;
  constexpr int TP = 32 * PW, SL = SV / TP, NB = TP + 96;
  constexpr int FS = NX == 2048 ? 2 * 1056 : (NX / 32) * 33;
  constexpr int NTW = NX == 2048 ? 2048 : NX;  // twiddle table entries
  static_assert(SV % TP == 0 && 1 + 2 * NPB <= 16 && NPB % FG == 0, "layout");
  constexpr unsigned kPoll = 1u << 22, kStageBytes = SV * sizeof(float4);
  extern __shared__ __align__(128) unsigned char smem_a128[];
  float4* stage = reinterpret_cast<float4*>(smem_a128);  // [S][SV]
  C* P = reinterpret_cast<C*>(stage + S * SV);            // [NPB][3][FS]
  C* tw4 = P + NPB * 3 * FS;                               // [max(NTW, 1024)]
  unsigned long long* full =
      reinterpret_cast<unsigned long long*>(tw4 + (NTW > 1024 ? NTW : 1024));
  unsigned long long* empty = full + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  static_assert(PW == 8 && FG == 3, "role table");
  int kind, ridx;
  if constexpr (NX == 2048) {  // measured faster in warp order for 2048-point rows
    kind = w < PW ? 0 : w < PW + 3 * FG ? 1 : 2;
    ridx = w < PW ? w : w - PW;
  } else {
    multi_role(w, kind, ridx);
  }
  if (t == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], PW);
    }
    *abort_flag = 0;
    fence_proxy_async();
  }
  for (int i = t; i < NTW; i += blockDim.x) tw4[i] = tw4_g[i];
  __shared__ float ang_ce[KMAX], ang_se[KMAX];  // indexed by a run-time angle
  if (t == 0) {
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {  // constant indices: the parameters stay in place
      ang_ce[i] = ang.ce[i];
      ang_se[i] = ang.se[i];
    }
  }
  __syncthreads();
  const int nk = ang.n;
  const long long nmine =
      blockIdx.x < nrows ? (nrows - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int per_row = pp.c;

  if (kind == 2) {  // producer warp, one lane (as in k_pol_fft4s_tma)
    if (lane != 0) return;
    // stage g = (row rr, segment h, component j), j fastest
    const int G = (int)nmine * H * per_row;
    int g = 0, slot = 0, k = 0, j = 0, h = 0;
    long long row = blockIdx.x;
    for (; g < G; ++g) {
      if (k > 0 && !mbar_wait_bounded(&empty[slot], (unsigned)((k - 1) & 1), poll)) {
        atomicOr(err, 1);
        *abort_flag = 1;
        break;
      }
      mbar_expect_tx(&full[slot], kStageBytes);
      bulk_g2s(stage + slot * SV, M + (size_t)j * N + (size_t)row * NX + h * SV, kStageBytes,
               &full[slot]);
      if (++slot == S) slot = 0, ++k;
      if (++j == per_row) {
        j = 0;
        if (++h == H) h = 0, row += gridDim.x;
      }
    }
    for (int d = g - 1; d >= 0 && d >= g - S; --d)
      mbar_wait_bounded(&full[d % S], (unsigned)((d / S) & 1), kPoll);
    return;
  }

  if (kind == 0) {  // polarisation warps; pt: this thread's index among them
    const int pt = ridx * 32 + lane;
    bool failed = false;
    int slot = 0, ph = 0;
    for (int rr = 0; rr < (int)nmine; ++rr) {
      for (int h = 0; h < H; ++h) {
        TAcc acc[SL];
#pragma unroll
        for (int sl = 0; sl < SL; ++sl) tacc_zero(acc[sl]);
        for (int j = 0; j < per_row; ++j) {
          const int cs = slot, cph = ph;
          if (++slot == S) slot = 0, ph ^= 1;
          failed = failed || __any_sync(0xffffffffu, *abort_flag != 0);
          if (failed) break;
          if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[cs], (unsigned)cph, poll))) {
            failed = true;
            atomicOr(err, 1);
            *abort_flag = 1;
            break;
          }
          const float4* st = stage + cs * SV;
          float4 cur[SL];
#pragma unroll
          for (int sl = 0; sl < SL; ++sl) cur[sl] = st[pt + sl * TP];
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[cs]);
#pragma unroll
          for (int sl = 0; sl < SL; ++sl)
            tacc_add(acc[sl], cur[sl].x, cur[sl].y, cur[sl].z, cur[sl].w, pp, j);
        }
        // (sum v^2 - 1) first, then the small optical part (FP32 accuracy);
        // everything divided by 4 pi once per voxel
        const float inv = float(1.0 / kFourPi);
#pragma unroll
        for (int sl = 0; sl < SL; ++sl) {
          acc[sl].aw = ((acc[sl].aw - 1.f) + acc[sl].as[0]) * inv;
          acc[sl].as[1] *= inv;
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            acc[sl].t[q][0] *= inv;
            acc[sl].t[q][1] *= inv;
          }
        }
        // row buffer u = rr * nk + k holds angle k of row rr; with H > 1 all
        // nk buffers of the row stay open across its segments (nk <= NPB)
        for (int k = 0; k < nk; ++k) {
          const int u = rr * nk + k, i = u % NPB;
          if (h == 0 && u >= NPB) named_bar_sync(1 + NPB + i, NB);  // previous use done
          if (!failed) {
            C* Pi = P + i * 3 * FS + h * 1056;
            const float ce = ang_ce[k], se = ang_se[k];
#pragma unroll
            for (int sl = 0; sl < SL; ++sl) {
              const int e = pt + sl * TP;
              C out[3];
              p_from_tacc(acc[sl].aw, acc[sl].as[1], acc[sl].t, ce, se, pp.literal != 0, out);
              Pi[e] = out[0];
              Pi[FS + e] = out[1];
              Pi[2 * FS + e] = out[2];
            }
          }
          if (h == H - 1) named_bar_arrive(1 + i, NB);
        }
      }
    }
    return;
  }

  // transform warps: group fg, field f; buffers u = fg, fg + FG, ...
  const int fg = ridx / 3, f = ridx % 3;
  const int U = (int)nmine * nk;
  for (int u = fg; u < U; u += FG) {
    const int i = u % NPB;
    named_bar_sync(1 + i, NB);
    if (*abort_flag == 0) {
      const int rr = u / nk, k = u - rr * nk;
      const long long row = blockIdx.x + (long long)rr * gridDim.x;
      xfft_row<NX>(P + i * 3 * FS + f * FS, tw4,
                   p + (size_t)k * pstride + (size_t)f * N + (size_t)row * NX, lane, [&] {
                     if (u + NPB < U) named_bar_arrive(1 + NPB + i, NB);
                   });
    } else if (u + NPB < U) {
      named_bar_arrive(1 + NPB + i, NB);
    }
  }
}

// ------------------------------------------------------ z-first x pass
// Algorithm 1's 3-D FFT of p, z axis first.  Each detector pixel reads two
// q_z bins of the transform, b0 = floor(t) and b0 + 1 with t = q_z / dq_z
// (Eq. (Ewald)); q_z <= 0 on the sphere and falls as the in-plane |q|
// grows, so over all pixels of one energy the bins read are the cyclic run
// kb, kb + 1, ..., kb + ns - 1 (mod nz) that ends at bin 1.  The 3-D DFT is
// separable, so its z transform may come first; the nz - ns bins no pixel
// reads are then dropped before the x and y transforms, which run on ns
// planes instead of nz slices (P1 geometry, 5 nm voxels: ns = 36 of 128 at
// 270 eV, 30 at 320 eV).
//
// This pass forms p as k_pol_fft4s_tma_multi does (same roles, ring and
// arithmetic: the morphology sums once per voxel, then each angle's p) but
// over tiles of XW = 32 / R adjacent pixels of one row y by the whole stack
// nz = 32 R (1024 voxels, one 3-D tensor copy per component), transforms
// every pixel's z column and stores planes s < ns (bin kb + s mod nz) of
// angle k at out + k * kstride + f * fstride + s * nx * ny (+ y nx + x).
//
// Row buffers hold a field as XW lines of LS complex; sample z of line px
// sits at px * LS + zf_pos(z >> 5, z & 31).  The z transform is a
// decimation in frequency with nz = 32 R, n = n2 + 32 n1, k = R k2 + k1
// (n2, k2 < 32; n1, k1 < R):
//   X[R k2 + k1] = sum_n2 W32^(n2 k2) W_nz^(n2 k1) sum_n1 x[n2 + 32 n1] W_R^(n1 k1);
//   stage 1, in the polarisation warps: a thread's four voxels of one
//            pixel (e = pt + 256 sl) sit at z = z0 + (256 / XW) sl, so
//            for R = 4 they are the four n1 of n2 = z0 and for R = 2 the
//            two n1 of n2 = z0 (sl = 0, 2) and of n2 = z0 + 16 (sl = 1, 3):
//            the R-point DFT over n1 runs on each angle's p in registers,
//            and u[k1][n2] is stored where x[n2 + 32 k1] would sit,
//            zf_pos(k1, n2), so the buffer holds stage 1's output;
//   stage 2: transform-warp lane (px, k1) loads u[k1][0..32) times
//            W_nz^(n2 k1) (each twiddle used as it is read), does the
//            32-point DFT and stores X[R k2 + k1] over the same 32
//            positions, zf_pos(k1, k2);
// then the warp copies the ns kept bins of its XW lines out (XW adjacent
// pixels per plane row).  zf_pos(a, b) = 32 a + b, for R = 4 with b xor a
// (the low bits swizzled by a); with LS = 130 (R = 4) or nz + 1 that keeps
// the polarisation stores, stage 2 and the copy free of shared-memory bank
// conflicts (checked per half-warp for R = 1, 2, 4).
template <int R> struct ZfLayout {
  static constexpr int NZ = 32 * R, XW = 32 / R, LXW = R == 1 ? 5 : R == 2 ? 4 : 3;
  static constexpr int LS = R == 4 ? 130 : NZ + 1, FS = XW * LS;
};
template <int R> __device__ __forceinline__ int zf_pos(int a, int b) {
  return 32 * a + (R == 4 ? (b ^ a) : b);
}

// Stage 2 of the z transform of one field of a row buffer (stage 1 done by
// the polarisation warps as they store p).
template <int R>
__device__ __forceinline__ void zfft_lines(float2* F, const float2* twt, int lane) {
  using C = float2;
  using Lay = ZfLayout<R>;
  constexpr int XW = Lay::XW, LS = Lay::LS;
  const int px = lane & (XW - 1), r = lane >> Lay::LXW;  // r < R
  C* Ln = F + px * LS;
  // zf_pos(a, b) for b = 4 j + c is base[c] + 4 j with base[c] = 32 a +
  // (c xor a): R base addresses per lane and immediate offsets
  // (a = k1 = r, b = n2 or k2)
  C* b2[R];
#pragma unroll
  for (int c = 0; c < R; ++c) b2[c] = Ln + zf_pos<R>(r, c);
  const C* tw = twt + r;
  C v[32];
#pragma unroll
  for (int n2 = 0; n2 < 32; ++n2) {
    const C a = b2[n2 % R][n2 - n2 % R];
    v[n2] = (R > 1 && n2 > 0) ? cmul(a, tw[n2 * R]) : a;
  }
  dft32(v);
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) b2[k2 % R][k2 - k2 % R] = v[k2];
  __syncwarp();
}

// Roles of the 18 warps of the z-first pass for nz = 128.  The split was
// set when a transform warp also ran the z transform's first radix stage
// (~1.2x the per-tile work of a polarisation warp): over the four
// schedulers (warp index mod 4) Prod T T T P | P P P P P | T T T P
// | T T T P kept every scheduler within ~7 % of the mean, and each
// transform group (three consecutive indices) spans three schedulers: warps
// 0, 2, 3, 4, 6, 7, 8, 10, 11 transform (0..8), 16 produces, 1, 5, 9, 13,
// 17, 12, 14, 15 polarise (0..7).  (P1: x pass 72.8 -> 72.2 ms per energy;
// nz = 64 measured 3 % slower with it and keeps multi_role.)
__device__ __forceinline__ void zf_role(int w, int& kind, int& idx) {
  const int q = w & 3;
  if (w == 16) {
    kind = 2;
    idx = 0;
  } else if (w < 12 && q != 1) {
    kind = 1;
    idx = (w >> 2) * 3 + (q == 0 ? 0 : q - 1);
  } else {
    kind = 0;
    idx = q == 1 ? w >> 2 : w == 12 ? 5 : w - 8;
  }
}

template <int R, int S, int NPB, int PW, int FG, int KMAX>
__global__ void __launch_bounds__(32 * (PW + 3 * FG + 1), 1) k_pol_zfft_multi(
    const __grid_constant__ CUtensorMap tmap, int nx, long long npix, long long ntiles,
    PolParams<float> pp, XAngles ang, float2* __restrict__ out, long long kstride,
    long long fstride, int kb, int ns, const float2* __restrict__ twz_g,
    int* __restrict__ err, unsigned poll) {
  using C = float2;
  using Lay = ZfLayout<R>;
  constexpr int NZ = Lay::NZ, XW = Lay::XW, LXW = Lay::LXW, LS = Lay::LS, FS = Lay::FS;
  constexpr int SV = 1024, TP = 32 * PW, SL = SV / TP, NB = TP + 96;
  static_assert(KMAX <= kMaxXAngles && SV % TP == 0 && 1 + 2 * NPB <= 16 && NPB % FG == 0,
                "layout");
  static_assert(PW == 8 && FG == 3 && SL == 4, "role table, stage-1 voxel groups");
  constexpr unsigned kPoll = 1u << 22, kStageBytes = SV * sizeof(float4);
  extern __shared__ __align__(128) unsigned char smem_a128[];
  float4* stage = reinterpret_cast<float4*>(smem_a128);  // [S][NZ][XW] voxels
  C* P = reinterpret_cast<C*>(stage + S * SV);            // [NPB][3][FS]
  C* twt = P + NPB * 3 * FS;                              // [32][R]: W_nz^(n2 k1)
  unsigned long long* full = reinterpret_cast<unsigned long long*>(twt + 32 * R);
  unsigned long long* empty = full + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  int kind, ridx;
  if constexpr (R == 4)
    zf_role(w, kind, ridx);
  else
    multi_role(w, kind, ridx);
  if (t == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], PW);
    }
    *abort_flag = 0;
    fence_proxy_async();
  }
  for (int i = t; i < 32 * R; i += blockDim.x) twt[i] = twz_g[(i / R) * (i % R)];
  __shared__ float ang_ce[KMAX], ang_se[KMAX];  // indexed by a run-time angle
  if (t == 0) {
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {  // constant indices: the parameters stay in place
      ang_ce[i] = ang.ce[i];
      ang_se[i] = ang.se[i];
    }
  }
  __syncthreads();
  const int nk = ang.n;
  const long long nmine =
      blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int per_row = pp.c;
  const int nxt = nx >> LXW;  // tiles per row y

  if (kind == 2) {  // producer lane: stage g = (tile rr, component j), j fastest
    if (lane != 0) return;
    const int G = (int)nmine * per_row;
    int g = 0, slot = 0, k = 0, j = 0;
    long long tile = blockIdx.x;
    for (; g < G; ++g) {
      if (k > 0 && !mbar_wait_bounded(&empty[slot], (unsigned)((k - 1) & 1), poll)) {
        atomicOr(err, 1);
        *abort_flag = 1;
        break;
      }
      const int y = (int)(tile / nxt), xb = (int)(tile - (long long)y * nxt);
      mbar_expect_tx(&full[slot], kStageBytes);
      tma_load_3d(stage + slot * SV, &tmap, xb * XW * 4, y, j * NZ, &full[slot]);
      if (++slot == S) slot = 0, ++k;
      if (++j == per_row) j = 0, tile += gridDim.x;
    }
    for (int d = g - 1; d >= 0 && d >= g - S; --d)
      mbar_wait_bounded(&full[d % S], (unsigned)((d / S) & 1), kPoll);
    return;
  }

  if (kind == 0) {  // polarisation warps; pt: this thread's index among them
    const int pt = ridx * 32 + lane;
    bool failed = false;
    int slot = 0, ph = 0;
    for (int rr = 0; rr < (int)nmine; ++rr) {
      TAcc acc[SL];
#pragma unroll
      for (int sl = 0; sl < SL; ++sl) tacc_zero(acc[sl]);
      for (int j = 0; j < per_row; ++j) {
        const int cs = slot, cph = ph;
        if (++slot == S) slot = 0, ph ^= 1;
        failed = failed || __any_sync(0xffffffffu, *abort_flag != 0);
        if (failed) break;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[cs], (unsigned)cph, poll))) {
          failed = true;
          atomicOr(err, 1);
          *abort_flag = 1;
          break;
        }
        const float4* st = stage + cs * SV;
        float4 cur[SL];
#pragma unroll
        for (int sl = 0; sl < SL; ++sl) cur[sl] = st[pt + sl * TP];
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[cs]);
#pragma unroll
        for (int sl = 0; sl < SL; ++sl)
          tacc_add(acc[sl], cur[sl].x, cur[sl].y, cur[sl].z, cur[sl].w, pp, j);
      }
      const float inv = float(1.0 / kFourPi);
#pragma unroll
      for (int sl = 0; sl < SL; ++sl) {
        acc[sl].aw = ((acc[sl].aw - 1.f) + acc[sl].as[0]) * inv;
        acc[sl].as[1] *= inv;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          acc[sl].t[q][0] *= inv;
          acc[sl].t[q][1] *= inv;
        }
      }
      for (int k = 0; k < nk; ++k) {
        const int u = rr * nk + k, i = u % NPB;
        if (u >= NPB) named_bar_sync(1 + NPB + i, NB);  // previous use done
        if (!failed) {
          C* Pi = P + i * 3 * FS;
          const float ce = ang_ce[k], se = ang_se[k];
          C o[SL][3];
#pragma unroll
          for (int sl = 0; sl < SL; ++sl)
            p_from_tacc(acc[sl].aw, acc[sl].as[1], acc[sl].t, ce, se, pp.literal != 0, o[sl]);
          // stage 1 of the z transform: sl = g + (4 / R) n1 holds n1 of one n2
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            if constexpr (R == 4) {
              dft4(o[0][f], o[1][f], o[2][f], o[3][f]);
            } else if constexpr (R == 2) {
              dft2(o[0][f], o[2][f]);
              dft2(o[1][f], o[3][f]);
            }
          }
#pragma unroll
          for (int sl = 0; sl < SL; ++sl) {
            // voxel (z, px) of the tile; after stage 1 its slot holds k1 = n1
            const int e = pt + sl * TP, z = e >> LXW;
            const int at = (e & (XW - 1)) * LS + zf_pos<R>(z >> 5, z & 31);
            Pi[at] = o[sl][0];
            Pi[FS + at] = o[sl][1];
            Pi[2 * FS + at] = o[sl][2];
          }
        }
        named_bar_arrive(1 + i, NB);
      }
    }
    return;
  }

  // transform warps: group fg, field f; buffers u = fg, fg + FG, ...
  const int fg = ridx / 3, f = ridx % 3;
  const int U = (int)nmine * nk;
  const int cnt = ns * XW;
  for (int u = fg; u < U; u += FG) {
    const int i = u % NPB;
    named_bar_sync(1 + i, NB);
    if (*abort_flag == 0) {
      const int rr = u / nk, k = u - rr * nk;
      const long long tile = blockIdx.x + (long long)rr * gridDim.x;
      const int y = (int)(tile / nxt), x0 = (int)(tile - (long long)y * nxt) * XW;
      C* F = P + i * 3 * FS + f * FS;
      zfft_lines<R>(F, twt, lane);
      C* o = out + (size_t)k * kstride + (size_t)f * fstride + (size_t)y * nx + x0;
      for (int idx = lane; idx < cnt; idx += 32) {
        const int s = idx >> LXW, px = idx & (XW - 1), kz = (kb + s) & (NZ - 1);
        o[(size_t)s * npix + px] = F[px * LS + zf_pos<R>(kz & (R - 1), kz / R)];
      }
      __syncwarp();
    }
    if (u + NPB < U) named_bar_arrive(1 + NPB + i, NB);
  }
}

// x-FFT of contiguous rows of NX complex in place (the kept q_z planes of
// the z-first path): one warp per row, the row staged in shared memory in
// the layout xfft_row<NX> takes (2048 points: halves at 0 and 1056; every
// copy 16-byte aligned: rows of 8 NX bytes, FS and NTW even), then
// xfft_row's four-step transform writes it back.  tw_g: the table xfft_row
// uses (1024: W1024^(n1 k2) as [32][32]; 2048: that, then W2048^n, n < 1024;
// 512: W512^j).
template <int NX, int W>
__global__ void __launch_bounds__(32 * W) k_xfft_rows(float2* __restrict__ data, long long nrows,
                                                      const float2* __restrict__ tw_g) {
  using C = float2;
  constexpr int FS = NX == 2048 ? 2 * 1056 : (NX / 32) * 33;
  constexpr int NTW = NX == 2048 ? 2048 : NX == 1024 ? 1024 : 512;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* F = tw + NTW + (threadIdx.x >> 5) * FS;
  const int lane = threadIdx.x & 31;
  const long long row = (long long)blockIdx.x * W + (threadIdx.x >> 5);
  C* r = data + (size_t)row * NX;
  // the row goes to shared memory by asynchronous 16-byte copies (a lane
  // keeps all NX / 64 of its copies in flight, no registers held), issued
  // before the twiddle table's loads so that the two overlap
  if (row < nrows) {
#pragma unroll
    for (int j = 0; j < NX / 64; ++j) {
      const int n = 2 * (lane + 32 * j);
      cp_async_pair(F + (NX == 2048 && n >= 1024 ? n + 32 : n), r + n);
    }
  }
  for (int i = threadIdx.x; i < NTW; i += 32 * W) tw[i] = tw_g[i];
  __syncthreads();
  if (row >= nrows) return;
  cp_async_wait_all();
  __syncwarp();
  xfft_row<NX>(F, tw, r, lane, [] {});
}

// y pass: a tile of TX adjacent columns of one batch.  Thread (n1, col)
// loads rows n1 + 32 n2 straight from global memory (32 independent loads),
// transforms over n2 in registers, applies the twiddles and writes row k2 of
// a [32][32 x TX] shared tile whose row stride 33 TX keeps both the writes
// (32 consecutive elements) and the transposed reads (the TX-wide groups of
// a half-warp land on disjoint bank windows) free of bank conflicts; thread
// (k2, col) then transforms over n1 and stores rows k2 + 32 k1.
template <typename R, int TX>
__global__ void __launch_bounds__(32 * TX, (sizeof(R) == 4 && TX <= 8) ? 2 : 1) k_col_fft4s(typename RT<R>::C* __restrict__ data,
                                                          long long S, long long ntiles,
                                                          long long bdiv, long long stride_hi,
                                                          long long stride_lo, long long base_off,
                                                          const typename RT<R>::C* __restrict__ tw4_g) {
  using C = typename RT<R>::C;
  constexpr int T = 32 * TX, STR = 33 * TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [32][STR]
  C* tw4 = buf + 32 * STR;                   // [32][32]
  const long long tile = (long long)blockIdx.x % ntiles;
  const long long b = (long long)blockIdx.x / ntiles;
  C* base = data + base_off + (b / bdiv) * stride_hi + (b % bdiv) * stride_lo + tile * TX;
  const int col = threadIdx.x % TX, n1 = threadIdx.x / TX;
  C v[32];
#pragma unroll
  for (int n2 = 0; n2 < 32; ++n2) v[n2] = __ldcs(base + (size_t)(n1 + 32 * n2) * S + col);
  for (int i = threadIdx.x; i < 1024; i += T) tw4[i] = tw4_g[i];
  dft32(v);
  __syncthreads();  // twiddle table in place
#pragma unroll
  for (int k2 = 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], tw4[k2 * 32 + n1]);
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) buf[k2 * STR + n1 * TX + col] = v[k2];
  __syncthreads();
  const int k2 = n1;
#pragma unroll
  for (int m = 0; m < 32; ++m) v[m] = buf[k2 * STR + m * TX + col];
  dft32(v);
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) base[(size_t)(k2 + 32 * k1) * S + col] = v[k1];
}

// y pass with tensor-memory-access loads (FP32, ny = 1024): persistent CTAs,
// one per SM, each walking tiles of 8 columns x 1024 rows.  Thread 0 loads
// the next-but-one tile with four 3-D TMA boxes (8 complex x 256 rows) into
// one of two input buffers while all threads transform the current one: the
// loads of a tile are in flight during the FFT of the previous tile.  The
// FFT is the four-step scheme of k_col_fft4s.  Waits are bounded; a timeout
// records *err, drains the copies in flight (bounded) and returns.
template <typename R>
__global__ void __launch_bounds__(256, 1) k_col_fft4s_tma(const __grid_constant__ CUtensorMap tmap,
                                                          typename RT<R>::C* __restrict__ data,
                                                          long long S, long long ntiles,
                                                          long long total, long long bdiv,
                                                          long long stride_hi, long long stride_lo,
                                                          const typename RT<R>::C* __restrict__ tw4_g,
                                                          int* __restrict__ err, unsigned poll) {
  using C = typename RT<R>::C;
  constexpr int TX = 8, T = 256, STR = 33 * TX, TILE = 1024 * TX;
  constexpr unsigned kPoll = 1u << 22;
  extern __shared__ __align__(128) unsigned char smem_a128[];
  C* in = reinterpret_cast<C*>(smem_a128);  // [2][1024][TX], dense (TMA boxes)
  C* tr = in + 2 * TILE;                    // [32][STR]
  C* tw4 = tr + 32 * STR;                   // [32][32]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(tw4 + 1024);
  const int t = threadIdx.x, col = t % TX, n1 = t / TX;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async();
  }
  for (int i = t; i < 1024; i += T) tw4[i] = tw4_g[i];
  __syncthreads();
  auto issue = [&](long long tile_id, int b) {
    const int ti = (int)(tile_id % ntiles), bb = (int)(tile_id / ntiles);
    mbar_expect_tx(&bar[b], TILE * sizeof(C));
#pragma unroll
    for (int q = 0; q < 4; ++q)
      tma_load_3d(in + b * TILE + q * 256 * TX, &tmap, ti * 2 * TX, q * 256, bb, &bar[b]);
  };
  if (t == 0) {
    if (blockIdx.x < total) issue(blockIdx.x, 0);
    if (blockIdx.x + gridDim.x < total) issue(blockIdx.x + gridDim.x, 1);
  }
  int i = 0;
  for (long long tid = blockIdx.x; tid < total; tid += gridDim.x, ++i) {
    const int b = i & 1;
    const bool ok = mbar_wait_bounded(&bar[b], (i >> 1) & 1, poll);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicOr(err, 1);
        for (int d = 0; d < 2; ++d)
          if (tid + d * gridDim.x < total) mbar_wait_bounded(&bar[(i + d) & 1], ((i + d) >> 1) & 1, kPoll);
      }
      return;
    }
    const C* src = in + b * TILE;
    C v[32];
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) v[n2] = src[(n1 + 32 * n2) * TX + col];
    dft32(v);
#pragma unroll
    for (int k2 = 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], tw4[k2 * 32 + n1]);
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) tr[k2 * STR + n1 * TX + col] = v[k2];
    __syncthreads();  // input buffer b consumed, transpose complete
    if (t == 0 && tid + 2 * gridDim.x < total) {
      fence_proxy_async();
      issue(tid + 2 * gridDim.x, b);
    }
    const int k2 = n1;
#pragma unroll
    for (int m = 0; m < 32; ++m) v[m] = tr[k2 * STR + m * TX + col];
    dft32(v);
    const long long ti = tid % ntiles, bb = tid / ntiles;
    C* base = data + (bb / bdiv) * stride_hi + (bb % bdiv) * stride_lo + ti * TX;
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) base[(size_t)(k2 + 32 * k1) * S + col] = v[k1];
    __syncthreads();  // the transpose buffer is rewritten by the next tile
  }
}

// Plain 1024-point row FFTs, one warp per row (four-step 32 x 32): lane n1
// loads the samples n1 + 32 n2 straight from global memory (32 coalesced
// loads in flight per lane), transforms over n2 in registers, twiddles,
// transposes through a padded 32 x 33 shared tile, transforms over n1 and
// stores X[k2 + 32 k1] (coalesced over k2).  src -> dst, may be in place.
template <typename R, int W>
__global__ void __launch_bounds__(32 * W) k_row_fft4s(const typename RT<R>::C* src,
                                                      typename RT<R>::C* dst, long long nrows,
                                                      const typename RT<R>::C* __restrict__ tw4_g) {
  using C = typename RT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw4 = reinterpret_cast<C*>(smem_raw);  // [32][32]
  C* F = tw4 + 1024 + (threadIdx.x >> 5) * (32 * 33);
  for (int i = threadIdx.x; i < 1024; i += 32 * W) tw4[i] = tw4_g[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long row = (long long)blockIdx.x * W + (threadIdx.x >> 5);
  if (row >= nrows) return;
  const C* in = src + (size_t)row * 1024 + lane;
  C v[32];
#pragma unroll
  for (int n2 = 0; n2 < 32; ++n2) v[n2] = in[32 * n2];
  dft32(v);
#pragma unroll
  for (int k2 = 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], tw4[k2 * 32 + lane]);
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) F[k2 * 33 + lane] = v[k2];
  __syncwarp();
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) v[n1] = F[lane * 33 + n1];
  dft32(v);
  C* out = dst + (size_t)row * 1024 + lane;
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) out[32 * k1] = v[k1];
}

// Plain row FFTs along x (no polarisation): the x pass of rsx_fft3d and of
// the linearity path; rows are read from src and written to p (src = p for
// in place).
template <typename R, int T, int EC>
__global__ void __launch_bounds__(T) k_row_fft(const typename RT<R>::C* src,
                                               typename RT<R>::C* p, int lognx, long long nrows,
                                               const typename RT<R>::C* __restrict__ twx,
                                               int tw_in_smem) {
  using C = typename RT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tws = buf + padded(EC);
  const int nx = 1 << lognx;
  const int ROWS = EC >> lognx;
  const long long row0 = (long long)blockIdx.x * ROWS;
  const long long rl = nrows - row0;
  const int rows_here = rl < ROWS ? (int)rl : ROWS;
  const int nel = rows_here << lognx;
  C* base = p + ((size_t)row0 << lognx);
  const C* sbase = src + ((size_t)row0 << lognx);
  if (tw_in_smem)
    for (int i = threadIdx.x; i < nx; i += T) tws[i] = twx[i];
  for (int e = threadIdx.x; e < nel; e += T) buf[padi(e)] = sbase[e];
  __syncthreads();
  const C* tw = tw_in_smem ? tws : twx;
  block_fft<R, EC, T, false>(buf, lognx, ROWS, -1, nx, 1, tw);
  for (int e = threadIdx.x; e < nel; e += T) base[e] = buf[padi(e)];
}

// Column FFTs: element i of column col of batch b sits at
//   data[off(b) + i * S + tile * TX + col],  i < L = 2^logL,
//   off(b) = base + (b / bdiv) * stride_hi + (b % bdiv) * stride_lo
// (batches = (component, z-slice) pairs for y, components for z).  One CTA
// transforms TX = 2^logTX adjacent columns (coalesced rows of TX complex
// values) of one batch; the tile arrives by cp.async, NLD copies per thread
// in flight, without passing registers.
template <typename R, int T, int EC, int LOGL, int MINB = 3>
__global__ void __launch_bounds__(T, MINB) k_col_fft(typename RT<R>::C* __restrict__ data, int logL_rt,
                                               long long S, int logTX_rt, long long ntiles,
                                               long long bdiv, long long stride_hi,
                                               long long stride_lo, long long base_off,
                                               const typename RT<R>::C* __restrict__ tw_g,
                                               int tw_in_smem) {
  using C = typename RT<R>::C;
  constexpr int NLD = EC / T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [L][TX], padded
  C* tws = buf + padded(EC);
  // with LOGL fixed, TX = EC / L is fixed too
  const int logL = LOGL >= 0 ? LOGL : logL_rt;
  const int logTX = LOGL >= 0 ? ilog2_ct(EC >> (LOGL >= 0 ? LOGL : 0)) : logTX_rt;
  const int L = 1 << logL;
  const int TX = 1 << logTX;
  const long long tile = (long long)blockIdx.x % ntiles;
  const long long b = (long long)blockIdx.x / ntiles;
  C* base = data + base_off + (b / bdiv) * stride_hi + (b % bdiv) * stride_lo + tile * TX;
  if (tw_in_smem)
    for (int i = threadIdx.x; i < L; i += T) tws[i] = tw_g[i];
  const int nel = L << logTX;
#pragma unroll
  for (int it = 0; it < NLD; ++it) {
    const int e = threadIdx.x + it * T;
    if (e < nel) cp_async_elem(buf + padi(e), base + (size_t)(e >> logTX) * S + (e & (TX - 1)));
  }
  cp_async_wait_all();
  __syncthreads();
  const C* tw = tw_in_smem ? tws : tw_g;
  if constexpr (LOGL >= 0)
    block_fft_ct<R, LOGL, (EC >> LOGL), 1, (EC >> LOGL), T, true>(buf, tw);
  else
    block_fft<R, EC, T, true>(buf, logL, TX, logTX, 1, TX, tw);
#pragma unroll
  for (int it = 0; it < NLD; ++it) {
    const int e = threadIdx.x + it * T;
    if (e < nel) base[(size_t)(e >> logTX) * S + (e & (TX - 1))] = buf[padi(e)];
  }
}

// 2048-point column FFTs (FP32): one CTA of 64 TX threads per tile of TX
// adjacent columns of one batch.  2048 = 64 x 32 with n = n1 + 64 n2 and
// k = k2 + 32 k1:
//   X[k2 + 32 k1] = sum_n1 W64^(n1 k1) W2048^(n1 k2) sum_n2 x[n1 + 64 n2] W32^(n2 k2).
// Stage 1: thread (n1, col) loads its 32 samples straight from global memory
// (32 loads in flight), does the 32-point DFT over n2 in registers, applies
// W2048^(n1 k2) and writes T[k2][n1][col] (k2 rows padded by TX elements, so
// the stage-2 reads of the k2 rows a half-warp covers fall in different
// banks).  Stage 2: threads (k2, col, h) and (k2, col, 1 - h), lanes 16
// apart, take the even (h = 0) and odd (h = 1) n1 of row k2: a 32-point DFT
// each, the odd half times W64^k, and one shuffle exchange leaves
// X[k2 + 32 k] on the h = 0 lane and X[k2 + 32 (k + 32)] on the h = 1 lane.
// tw[j] = W2048^j.
template <int TX>
__global__ void __launch_bounds__(64 * TX, 8 / TX) k_col_fft2k(float2* __restrict__ data,
                                                                long long S, long long ntiles,
                                                                long long bdiv, long long stride_hi,
                                                                long long stride_lo,
                                                                long long base_off,
                                                                const float2* __restrict__ tw_g) {
  using C = float2;
  static_assert(TX == 4 || TX == 8, "tile width");
  constexpr int T = 64 * TX, KS = 64 * TX + TX;  // threads; row stride of T (k2)
  constexpr int LT = 5 - (TX == 8 ? 3 : 2);      // log2(32 / TX)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Tm = reinterpret_cast<C*>(smem_raw);  // [32][KS]
  C* tw = Tm + 32 * KS;                    // [2048]
  const long long tile = (long long)blockIdx.x % ntiles;
  const long long b = (long long)blockIdx.x / ntiles;
  C* base = data + base_off + (b / bdiv) * stride_hi + (b % bdiv) * stride_lo + tile * TX;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  // stage 1: col = lane mod TX, n1 = (32 / TX) w + lane / TX
  {
    const int col = lane & (TX - 1), n1 = (w << LT) + lane / TX;
    C v[32];
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) v[n2] = __ldcs(base + (size_t)(n1 + 64 * n2) * S + col);
    for (int i = t; i < 2048; i += T) tw[i] = tw_g[i];
    dft32(v);
    __syncthreads();  // twiddle table in place
#pragma unroll
    for (int k2 = 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], tw[n1 * k2]);
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) Tm[k2 * KS + n1 * TX + col] = v[k2];
  }
  __syncthreads();
  // stage 2: col = lane mod TX, k2 = (16 / TX) w + (lane / TX mod 16 / TX), h = lane / 16
  const int col = lane & (TX - 1), k2 = w * (16 / TX) + ((lane / TX) & (16 / TX - 1)),
            h = lane >> 4;
  C v[32];
#pragma unroll
  for (int m = 0; m < 32; ++m) v[m] = Tm[k2 * KS + (2 * m + h) * TX + col];
  dft32(v);
  C* out = base + (size_t)(k2 + 1024 * h) * S + col;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const C mine = h ? cmul(v[k], tw[32 * k]) : v[k];  // E[k], or W64^k O[k]
    C other;
    other.x = __shfl_xor_sync(0xffffffffu, mine.x, 16);
    other.y = __shfl_xor_sync(0xffffffffu, mine.y, 16);
    out[(size_t)(32 * k) * S] = h ? csub(other, mine) : cadd(mine, other);
  }
}

// ------------------------------------------------ general-size transforms
// Up to kAnyMaxPass radices whose product is the transform length.
constexpr int kAnyMaxPass = 24;
struct AnyPlan {
  int n, np;
  int rad[kAnyMaxPass];
};

__device__ __forceinline__ long long any_line_start(const AnyLines& ln, long long l) {
  const long long b = l / ln.W, x = l - b * ln.W;
  return ln.base + (b / ln.bdiv) * ln.stride_hi + (b % ln.bdiv) * ln.stride_lo + x * ln.xstride;
}

// lpc lines per CTA, loaded whole into shared memory (buffer A), then the
// plan's passes alternate between A and B (the Stockham scheme of
// rsx_device.cuh with any radix), and the spectra are stored back.
// lines_fast: consecutive threads take consecutive lines (columns, whose
// lines are adjacent in memory) rather than consecutive elements (rows).
template <typename R>
__global__ void __launch_bounds__(256) k_fft_any(const typename RT<R>::C* src,
                                                 typename RT<R>::C* dst, AnyPlan plan, AnyLines ln,
                                                 int lpc, int lines_fast,
                                                 const typename RT<R>::C* __restrict__ tw_g) {
  using C = typename RT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = plan.n;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + (size_t)lpc * n;
  C* tw = B + (size_t)lpc * n;
  const long long l0 = (long long)blockIdx.x * lpc;
  const int nl = ln.nlines - l0 < lpc ? (int)(ln.nlines - l0) : lpc;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = tw_g[i];
  const int tot = nl * n;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int t = lines_fast ? e % nl : e / n, i = lines_fast ? e / nl : e % n;
    A[t * n + i] = src[any_line_start(ln, l0 + t) + (long long)i * ln.estride];
  }
  __syncthreads();
  C* x = A;
  C* y = B;
  int Ns = 1;
  for (int ps = 0; ps < plan.np; ++ps) {
    const int rad = plan.rad[ps], nb = n / rad;
    const bool general = rad != 2 && rad != 3 && rad != 4 && rad != 5 && rad != 7 && rad != 8 &&
                         rad != 16;
    if (general) {
      // other primes: one thread per output of a butterfly (O(rad) each)
      const int total = nl * nb * rad;
      for (int it = threadIdx.x; it < total; it += blockDim.x) {
        const int r = it % rad, q = it / rad;
        const int t = lines_fast ? q % nl : q / nb, j = lines_fast ? q / nl : q % nb;
        any_output_prime(x + t * n, y + t * n, j, r, rad, n, Ns, tw);
      }
    } else {
      const int total = nl * nb;
      for (int it = threadIdx.x; it < total; it += blockDim.x) {
        const int t = lines_fast ? it % nl : it / nb, j = lines_fast ? it / nl : it % nb;
        const C* xl = x + t * n;
        C* yl = y + t * n;
        switch (rad) {
          case 2: any_butterfly<2>(xl, yl, j, n, Ns, tw); break;
          case 3: any_butterfly<3>(xl, yl, j, n, Ns, tw); break;
          case 4: any_butterfly<4>(xl, yl, j, n, Ns, tw); break;
          case 5: any_butterfly<5>(xl, yl, j, n, Ns, tw); break;
          case 7: any_butterfly<7>(xl, yl, j, n, Ns, tw); break;
          case 8: any_butterfly<8>(xl, yl, j, n, Ns, tw); break;
          default: any_butterfly<16>(xl, yl, j, n, Ns, tw); break;
        }
      }
    }
    __syncthreads();
    C* tmp = x;
    x = y;
    y = tmp;
    Ns *= rad;
  }
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int t = lines_fast ? e % nl : e / n, i = lines_fast ? e / nl : e % n;
    dst[any_line_start(ln, l0 + t) + (long long)i * ln.estride] = x[t * n + i];
  }
}

// Direct DFT along z for any nz (out of place): out[k][m][pix] =// Direct DFT along z for any nz (out of place): out[k][m][pix] =
//   sum_z in[k][z][pix] exp(-2 pi i m z / nz).
template <typename R>
__global__ void k_dft_z(const typename RT<R>::C* __restrict__ in, typename RT<R>::C* __restrict__ out,
                        long long npix, int nz, const typename RT<R>::C* __restrict__ twz) {
  using C = typename RT<R>::C;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = 3 * npix * nz;
  if (t >= total) return;
  const long long pix = t % npix;
  const int m = (int)((t / npix) % nz);
  const int k = (int)(t / (npix * nz));
  const size_t N = (size_t)npix * nz;
  const C* src = in + k * N + pix;
  C acc = RT<R>::mk(0, 0);
  int idx = 0;
  for (int z = 0; z < nz; ++z) {
    acc = cadd(acc, cmul(src[(size_t)z * npix], twz[idx]));
    idx += m;
    if (idx >= nz) idx -= nz;
  }
  out[k * N + (size_t)m * npix + pix] = acc;
}

// Position in fftshift order (q = 0 at (ny / 2, nx / 2)) of the pixel with
// FFT-order index pix = my nx + mx, for any nx and ny.
__device__ __forceinline__ size_t shifted_pixel(long long pix, int nx, int ny) {
  const int my = (int)(pix / nx), mx = (int)(pix - (long long)my * nx);
  int sy = my + ny / 2, sx = mx + nx / 2;
  if (sy >= ny) sy -= ny;
  if (sx >= nx) sx -= nx;
  return (size_t)sy * nx + sx;
}

// --------------------------------------------------------------- geometry
// Eq. (Ewald) per pixel, in double: q from the FFT index (FFT order),
// q_z = -k + sqrt(k^2 - q_x^2 - q_y^2), t = q_z / dq_z, bins floor(t) and
// floor(t) + 1 (periodic), weight w = t - floor(t) on the upper bin.
// b0idx (optional): the lower bin alone, 0 off the sphere, for the fused
// y+z passes' per-tile tables (2 bytes per pixel instead of a 32-byte record).
template <typename R>
__global__ void k_geometry(Geo<R>* __restrict__ geo, int nx, int ny, int nz, double voxel_nm,
                           double k, unsigned short* __restrict__ b0idx) {
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= (long long)nx * ny) return;
  const int my = (int)(pix / nx), mx = (int)(pix - (long long)my * nx);
  const int fx = mx < (nx + 1) / 2 ? mx : mx - nx;
  const int fy = my < (ny + 1) / 2 ? my : my - ny;
  const double two_pi = 6.283185307179586476925286766559;
  const double qx = two_pi * fx / (nx * voxel_nm);
  const double qy = two_pi * fy / (ny * voxel_nm);
  const double rad = k * k - qx * qx - qy * qy;
  Geo<R> g;
  if (rad < 0.0) {
    g.b0 = g.b1 = -1;
    g.w = g.rx = g.ry = g.rz = g.k4 = R(0);
    geo[pix] = g;
    if (b0idx) b0idx[pix] = 0;
    return;
  }
  const double qz = -k + sqrt(rad);
  const double dqz = two_pi / (nz * voxel_nm);
  const double t = qz / dqz;
  const double z0 = floor(t);
  const double w = t - z0;
  long long i0 = (long long)z0 % nz;
  if (i0 < 0) i0 += nz;
  long long i1 = i0 + 1;
  if (i1 >= nz) i1 -= nz;
  const double kz = k + qz;
  const double kmag2 = qx * qx + qy * qy + kz * kz;
  const double kmag = sqrt(kmag2);
  g.b0 = (int)i0;
  g.b1 = (int)i1;
  g.w = (R)w;
  g.rx = (R)(qx / kmag);
  g.ry = (R)(qy / kmag);
  g.rz = (R)(kz / kmag);
  g.k4 = (R)(kmag2 * kmag2);
  geo[pix] = g;
  if (b0idx) b0idx[pix] = (unsigned short)i0;
}

// ------------------------------------------------------------------- Ewald
// |(I - r r) v|^2 = sum_k |v_k - r_k (r . v)|^2 for one bin.
template <typename R>
__device__ __forceinline__ R proj_norm2(const typename RT<R>::C v[3], R rx, R ry, R rz) {
  const R sr = rx * v[0].x + ry * v[1].x + rz * v[2].x;
  const R si = rx * v[0].y + ry * v[1].y + rz * v[2].y;
  const R y0r = v[0].x - rx * sr, y0i = v[0].y - rx * si;
  const R y1r = v[1].x - ry * sr, y1i = v[1].y - ry * si;
  const R y2r = v[2].x - rz * sr, y2i = v[2].y - rz * si;
  return y0r * y0r + y0i * y0i + y1r * y1r + y1i * y1i + y2r * y2r + y2i * y2i;
}

// Two adjacent pixels of one row, loaded as one 16-byte vector in FP32.
__device__ __forceinline__ void ld2(const float2* p, float2& a, float2& b) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(p));
  a = make_float2(q.x, q.y);
  b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void ld2(const double2* p, double2& a, double2& b) {
  a = __ldg(p);
  b = __ldg(p + 1);
}

template <typename R>
__device__ __forceinline__ R ewald_value(const Geo<R>& g, const typename RT<R>::C a0[3],
                                         const typename RT<R>::C a1[3]) {
  const R x0 = proj_norm2<R>(a0, g.rx, g.ry, g.rz);
  const R x1 = proj_norm2<R>(a1, g.rx, g.ry, g.rz);
  return g.k4 * ((R(1) - g.w) * x0 + g.w * x1);
}

// Full p~ given: read the two bins of each pixel (one thread per pixel).
template <typename R>
__global__ void __launch_bounds__(256) k_ewald_full(const typename RT<R>::C* __restrict__ p, int nx,
                                                    int ny, int nz, const Geo<R>* __restrict__ geo,
                                                    R* __restrict__ img) {
  using C = typename RT<R>::C;
  const long long npix = (long long)nx * ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  R* dst = img + shifted_pixel(pix, nx, ny);
  const Geo<R> g = geo[pix];
  if (g.b0 < 0) {
    *dst = R(0);
    return;
  }
  const size_t N = (size_t)npix * nz;
  C a0[3], a1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    a0[k] = p[k * N + (size_t)g.b0 * npix + pix];
    a1[k] = p[k * N + (size_t)g.b1 * npix + pix];
  }
  *dst = ewald_value<R>(g, a0, a1);
}

// Hot path: p holds x/y-transformed slices P(z).  Each thread takes two
// adjacent pixels of a row and evaluates the two q_z bins each needs,
//   p~(b) = sum_z P(z) exp(-2 pi i b z / nz),
// reading ZB slices' worth of vector loads before accumulating them.  The
// constant left out of p before the FFT returns at q = 0 as N * dc.
template <typename R, int ZB>
__global__ void __launch_bounds__(256) k_ewald_pruned(const typename RT<R>::C* __restrict__ p,
                                                      int nx, int ny, int nz,
                                                      const Geo<R>* __restrict__ geo,
                                                      const typename RT<R>::C* __restrict__ twz_g,
                                                      int tw_in_smem, R dc0, R dc1, R dc2,
                                                      R* __restrict__ img) {
  using C = typename RT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tws = reinterpret_cast<C*>(smem_raw);
  if (tw_in_smem) {
    for (int i = threadIdx.x; i < nz; i += blockDim.x) tws[i] = twz_g[i];
    __syncthreads();
  }
  const C* twz = tw_in_smem ? tws : twz_g;
  const long long npix = (long long)nx * ny;
  const long long pix0 = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (pix0 >= npix) return;
  const size_t N = (size_t)npix * nz;
  Geo<R> g[2];
  g[0] = geo[pix0];
  g[1] = geo[pix0 + 1];
  C a0[2][3], a1[2][3];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < 3; ++k) a0[q][k] = a1[q][k] = RT<R>::mk(0, 0);
  const bool any = g[0].b0 >= 0 || g[1].b0 >= 0;
  int i0[2] = {0, 0}, i1[2] = {0, 0};
  const int s0[2] = {g[0].b0 < 0 ? 0 : g[0].b0, g[1].b0 < 0 ? 0 : g[1].b0};
  const int s1[2] = {g[0].b1 < 0 ? 0 : g[0].b1, g[1].b1 < 0 ? 0 : g[1].b1};
  const C* src = p + pix0;
  int z = 0;
  if (any) {
    for (; z + ZB <= nz; z += ZB) {
      C v[ZB][3][2];
#pragma unroll
      for (int u = 0; u < ZB; ++u)
#pragma unroll
        for (int k = 0; k < 3; ++k) ld2(src + k * N + (size_t)(z + u) * npix, v[u][k][0], v[u][k][1]);
#pragma unroll
      for (int u = 0; u < ZB; ++u) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const C w0 = twz[i0[q]], w1 = twz[i1[q]];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            a0[q][k] = cadd(a0[q][k], cmul(v[u][k][q], w0));
            a1[q][k] = cadd(a1[q][k], cmul(v[u][k][q], w1));
          }
          i0[q] += s0[q];
          if (i0[q] >= nz) i0[q] -= nz;
          i1[q] += s1[q];
          if (i1[q] >= nz) i1[q] -= nz;
        }
      }
    }
    for (; z < nz; ++z) {
      C v[3][2];
#pragma unroll
      for (int k = 0; k < 3; ++k) ld2(src + k * N + (size_t)z * npix, v[k][0], v[k][1]);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const C w0 = twz[i0[q]], w1 = twz[i1[q]];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          a0[q][k] = cadd(a0[q][k], cmul(v[k][q], w0));
          a1[q][k] = cadd(a1[q][k], cmul(v[k][q], w1));
        }
        i0[q] += s0[q];
        if (i0[q] >= nz) i0[q] -= nz;
        i1[q] += s1[q];
        if (i1[q] >= nz) i1[q] -= nz;
      }
    }
  }
  if (pix0 == 0) {
    const R dcs[3] = {dc0, dc1, dc2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (g[0].b0 == 0) a0[0][k].x += dcs[k];
      if (g[0].b1 == 0) a1[0][k].x += dcs[k];
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const long long pix = pix0 + q;
    img[shifted_pixel(pix, nx, ny)] = g[q].b0 < 0 ? R(0) : ewald_value<R>(g[q], a0[q], a1[q]);
  }
}

// Stage-1 samples of the 2048-row fused pass: virtual column col of the
// 1024-point transforms is, for col < 4, a[r] = x[r] + x[r + 1024] and, for
// col >= 4, b[r] = (x[r] - x[r + 1024]) W2048^r of real column col mod 4
// (radix-2 decimation in frequency: X[2k] and X[2k + 1] are the 1024-point
// transforms of a and b).  With r = r0 + 64 m, W2048^r = W2048^r0 W32^m; the
// W32^m factor is applied here (a compile-time constant, selected per lane),
// W2048^r0 after the 16-point DFT.  xb holds the tile as [2048][4].
template <int M>
__device__ __forceinline__ void yz2k_load(const float2* xb, int r0, int c4, bool odd, float2* v) {
  if constexpr (M < 16) {
    const float2 x1 = xb[(r0 + 64 * M) * 4 + c4], x2 = xb[(r0 + 64 * M + 1024) * 4 + c4];
    const float2 a = cadd(x1, x2), d = csub(x1, x2);
    const float2 b = w32<M>(d);
    v[M].x = odd ? b.x : a.x;
    v[M].y = odd ? b.y : a.y;
    yz2k_load<M + 1>(xb, r0, c4, odd, v);
  }
}

// y-FFT fused with the pruned z transform (FP32, ny = 1024, nz a power of
// two up to 1024, nx a multiple of 16).  Work items are (field, pair of
// adjacent 8-column tiles); each has nz steps (its z-slices).  The items'
// steps are laid end to end and cut into one contiguous range of L >= nz
// steps per pair of persistent CTAs (blocks 2j and 2j + 1 take the even and
// the odd tile of the same steps, so the two 64-byte halves of every
// 128-byte row segment are read at about the same time: DRAM fetches whole
// lines).  Every CTA does the same number of steps; with L >= nz / 3 an item
// is split between at most four CTA pairs: the part that starts at z = 0
// goes to slot 0 of `part`, the others to slots 1-3 in order, and
// k_ewald_bins adds them.
//
// Per step the slice's 8 x 1024 tile arrives by 2-D tensor TMA (two
// buffers).  The four-step 32 x 32 FFT is split between the two halves of
// the block (hw = warp / 8, uniform per warp, so every twiddle below is a
// compile-time constant and no lane selects between two roles):
//  stage 1: half hw takes the samples n2 = 2m + hw of row n1 and stores
//           its 16-point DFT, the odd half times W32^k, to `tr`;
//  stage 2: thread (k2, hw) forms the stage-1 outputs X1[n1][k2] = E +- O'
//           for n1 = 2m + hw, applies W1024^(n1 k2), does its 16-point DFT
//           (odd half times W32^k) and swaps halves with its partner through
//           the input buffer it has just consumed;
// after which each thread holds 16 pixels (row k2 + 32 k1, k1 = 16 hw ..
// 16 hw + 15) and accumulates, across the item's z-slices, the two q_z bins
// b0 and b0 + 1 of Eq. (Ewald):
//   A0 += Y(z) W^(b0 z),  A1 += Y(z) W^(b0 z) W^z,  W = exp(-2 pi i / nz),
// with b0 per pixel from the energy's geometry (0 for pixels off the
// sphere, which k_ewald_bins zeroes).  The y-transformed slices are never
// written.  The input buffer is refilled (step + 2) once the swap has been
// read.  Waits are bounded as in k_col_fft4s_tma.
//
// Y2K: the same for ny = 2048.  A work item is (field, quad of adjacent
// 4-column tiles), blocks 4j .. 4j + 3 take the four tiles of the same
// steps (32-byte row segments, a 128-byte line per quad); each step's
// 4 x 2048 tile arrives in eight 256-row boxes and is read by stage 1 as the
// 8 virtual columns of two 1024-point transforms (yz2k_load: even outputs
// from columns 0-3, odd from 4-7), so the rest of the pass is unchanged;
// virtual pixel (row, col) is the real pixel (2 row + col / 4, 4 ti + col mod 4).
// tw2k: W2048^j (j < 64 used).
//
// SEL: the z-first path's planes instead of z-slices.  A field holds nz = ns
// planes (any count), plane s being bin (kb + s) mod (zmask + 1) of the z
// transform, already x-transformed; each pixel's two bins are planes
// sb = (b0 - kb) mod (zmask + 1) and sb + 1, so a step selects instead of
// accumulating: A0 = Y(sb), A1 = Y(sb + 1) (twz unused).
template <bool Y2K, bool SEL>
__global__ void __launch_bounds__(512, 1) k_yz_tma(const __grid_constant__ CUtensorMap tmap, int nx,
                                                   int nz, int nf, int ntiles, int L, int T,
                                                   const Geo<float>* __restrict__ geo,
                                                   const float2* __restrict__ twz_g,
                                                   const float2* __restrict__ tw4_g,
                                                   const float2* __restrict__ tw2k,
                                                   const unsigned short* __restrict__ b0idx,
                                                   float4* __restrict__ part, int* __restrict__ err,
                                                   unsigned poll, int kb, int zmask) {
  using C = float2;
  constexpr int TX = 8, TILE = 1024 * TX, STR = 33 * TX;
  constexpr int GRP = Y2K ? 4 : 2, LGRP = Y2K ? 2 : 1;  // blocks reading one line in lockstep
  constexpr unsigned kPoll = 1u << 22;
  extern __shared__ __align__(128) unsigned char smem_a128[];
  C* in = reinterpret_cast<C*>(smem_a128);  // [2][1024][TX], dense (TMA boxes)
  C* tr = in + 2 * TILE;                     // [32][STR]
  C* tw4 = tr + 32 * STR;                    // [32][32], symmetric
  C* twz = tw4 + 1024;                       // [nz]
  unsigned short* btab = reinterpret_cast<unsigned short*>(twz + nz);  // [1024][TX]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(btab + TILE);
  // SEL: each thread's 16 plane indices as bytes, [512][16] over the unused
  // twz (16-byte aligned), read as one 16-byte word per step
  unsigned char* btab8 = reinterpret_cast<unsigned char*>(twz);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int col = lane & 7, hw = w >> 3;
  const int q = (w & 7) * 4 + (lane >> 3);  // n1 in stage 1, k2 in stage 2
  // 32-bit step arithmetic (T < 2^31); nz and ntiles / GRP are powers of two
  const int s0 = (int)(blockIdx.x >> LGRP) * L;
  const int s1 = s0 + L < T ? s0 + L : T;
  if (s0 >= s1) return;
  const long long npix = (Y2K ? 2048LL : 1024LL) * nx;
  const int half = ntiles >> LGRP, lognz = __ffs(nz) - 1, loghalf = __ffs(half) - 1;
  const int mem = blockIdx.x & (GRP - 1);
  // Y2K: this lane's W2048^r0 (r0 = q + 32 hw) for the odd virtual columns
  const bool odd = Y2K && col >= 4;
  const C base2k = odd ? tw2k[q + 32 * hw] : make_float2(1.f, 0.f);
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async();
  }
  for (int i = t; i < 1024; i += 512) tw4[i] = tw4_g[i];
  if constexpr (!SEL)
    for (int i = t; i < nz; i += 512) twz[i] = twz_g[i];
  __syncthreads();
  // step st -> (work item, slice or plane z)
  auto split = [&](int st, int& item, int& z) {
    if constexpr (SEL) {
      item = st / nz;
      z = st - item * nz;
    } else {
      item = st >> lognz;
      z = st & (nz - 1);
    }
  };
  auto issue = [&](int st, int b) {
    int item, z;
    split(st, item, z);
    const int f = item >> loghalf, ti = GRP * (item & (half - 1)) + mem;
    mbar_expect_tx(&bar[b], TILE * sizeof(C));
    if constexpr (Y2K) {  // 4 columns (8 floats) x 2048 rows
#pragma unroll
      for (int k = 0; k < 8; ++k)
        tma_load_3d(in + b * TILE + k * 256 * 4, &tmap, ti * 8, k * 256, f * nz + z, &bar[b]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        tma_load_3d(in + b * TILE + k * 256 * TX, &tmap, ti * 2 * TX, k * 256, f * nz + z, &bar[b]);
    }
  };
  if (t == 0) {
    issue(s0, 0);
  }
  C acc0[16], acc1[16];
  int i = 0;
  for (int st = s0; st < s1; ++st, ++i) {
    const int b = i & 1;
    int item, z;
    split(st, item, z);
    const int ti = GRP * (item & (half - 1)) + mem;
    if (z == 0 || st == s0) {  // a new segment: this tile's bins, zero accumulators
      __syncthreads();  // the previous step's reads of the bins are done
      for (int e = t; e < TILE; e += 512) {
        const size_t pixel = Y2K ? (size_t)(2 * (e >> 3) + ((e & 7) >> 2)) * nx + ti * 4 + (e & 3)
                                 : (size_t)(e >> 3) * nx + ti * TX + (e & 7);
        const int bin = b0idx[pixel];
        if constexpr (SEL) {
          // virtual pixel (row, col) belongs to the stage-3 thread
          // (q, hw, col) with row = q + 512 hw + 32 k: byte k of its word
          const int row = e >> 3, rem = row & 511, qq = rem & 31;
          const int owner = ((row >> 9) * 8 + (qq >> 2)) * 32 + ((qq & 3) << 3) + (e & 7);
          btab8[owner * 16 + (rem >> 5)] = (unsigned char)((bin - kb) & zmask);
        } else {
          btab[e] = (unsigned short)bin;
        }
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) acc0[k] = acc1[k] = make_float2(0.f, 0.f);
    }
    const bool ok = mbar_wait_bounded(&bar[b], (i >> 1) & 1, poll);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicOr(err, 1);
        // only this step's load is in flight (the next one is issued later)
        mbar_wait_bounded(&bar[b], (i >> 1) & 1, kPoll);
      }
      return;
    }
    C* const xb = in + b * TILE;
    // stage 1: 16-point DFT of the samples n2 = 2m + hw of row n1 = q
    {
      C v[16];
      if constexpr (Y2K) {
        yz2k_load<0>(xb, q + 32 * hw, col & 3, odd, v);
      } else {
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = xb[(q + 32 * hw + 64 * m) * TX + col];
      }
      dft_reg<16>(v);
      if constexpr (Y2K) {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = cmul(v[k], base2k);
      }
      if (hw) w32_outputs<0>(v);
#pragma unroll
      for (int k = 0; k < 16; ++k) tr[(16 * hw + k) * STR + q * TX + col] = v[out_pos<16>(k)];
    }
    __syncthreads();  // stage-1 halves in tr, bins in place; xb consumed
    // the other buffer held the previous step, whose reads all came before
    // this barrier: load the next step into it
    if (t == 0 && st + 1 < s1) {
      fence_proxy_async();
      issue(st + 1, b ^ 1);
    }
    // stage 2: X1[n1][k2] = E +- O' (minus for k2 >= 16), times W1024^(n1 k2)
    C v[16];
    {
      const int k = q & 15;
      const bool upper = q >= 16;  // warp-uniform
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int n1 = 2 * m + hw;
        const C e = tr[k * STR + n1 * TX + col];
        const C o = tr[(16 + k) * STR + n1 * TX + col];
        v[m] = cmul(upper ? csub(e, o) : cadd(e, o), tw4[n1 * 32 + q]);
      }
      dft_reg<16>(v);
      if (hw) w32_outputs<0>(v);
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) xb[(16 * hw + k2) * 256 + q * TX + col] = v[out_pos<16>(k2)];
    }
    __syncthreads();  // halves swapped; every stage-2 read of tr is done
    {
      const C wz = SEL ? make_float2(1.f, 0.f) : twz[z];
      uint4 sb4 = make_uint4(0u, 0u, 0u, 0u);
      float2* sel0 = nullptr;  // SEL: slot 0 of this thread's pixel column, as float2 pairs
      if constexpr (SEL) {
        sb4 = reinterpret_cast<const uint4*>(btab8)[t];
        sel0 = reinterpret_cast<float2*>(
            part + (size_t)(item >> loghalf) * npix +
            (Y2K ? (size_t)(col >> 2) * nx + ti * 4 + (col & 3) : (size_t)ti * TX + col));
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const C mine = v[out_pos<16>(k)];
        const C other = xb[(16 * (1 - hw) + k) * 256 + q * TX + col];
        const C y = hw ? csub(other, mine) : cadd(mine, other);  // X[k2 + 32 (16 hw + k)]
        const int row = q + 512 * hw + 32 * k;
        if constexpr (SEL) {
          // each pixel's bins come from one plane each: stored as they pass
          const unsigned wd = k < 4 ? sb4.x : k < 8 ? sb4.y : k < 12 ? sb4.z : sb4.w;
          const int sb = (int)((wd >> (8 * (k & 3))) & 0xffu);
          float2* d = sel0 + 2 * (size_t)row * (Y2K ? 2 * nx : nx);
          if (sb == z) d[0] = y;
          if (sb + 1 == z) d[1] = y;
        } else {
          const int b0 = btab[row * TX + col];
          const C qq = cmul(y, twz[(b0 * z) & (nz - 1)]);
          acc0[k] = cadd(acc0[k], qq);
          acc1[k] = cadd(acc1[k], cmul(qq, wz));
        }
      }
      if (!SEL && (z == nz - 1 || st == s1 - 1)) {  // segment end: slot 0 if it began at z = 0
        // slot: this segment's place among the item's segments (0 if it
        // began at z = 0); L >= nz / 3 keeps it below kYzSlots
        const int item_start = st - z;
        const int slot = item_start >= s0 ? 0 : s0 / L - item_start / L;
        const int f = item >> loghalf;
        float4* dst = part + ((size_t)slot * nf + f) * npix +
                      (Y2K ? (size_t)(col >> 2) * nx + ti * 4 + (col & 3) : (size_t)ti * TX + col);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int row = q + 512 * hw + 32 * k;
          dst[(size_t)row * (Y2K ? 2 * nx : nx)] =
              make_float4(acc0[k].x, acc0[k].y, acc1[k].x, acc1[k].y);
        }
      }
    }
  }
}

// The fused y-FFT + q_z bins pass for ny = 512 (FP32, nx a multiple of 16,
// nz a power of two up to 1024).  Work items are (field, 16-column tile), so
// every row segment a tile reads is a whole 128-byte line; the items'
// z-slices are cut into equal contiguous ranges, one per persistent block
// (slots as in k_yz_tma).  512 = 16 x 32 with n = n1 + 16 n2 and
// k = k2 + 32 k1:
//  stage 1: half hw (warps 0-7 / 8-15) takes the samples n2 = 2m + hw of
//           row n1 (16 x 16 columns per half) and stores its 16-point DFT,
//           the odd half times W32^k;
//  stage 2: thread (k2, column) forms X1[n1][k2] = E +- O' for all 16 n1,
//           applies W512^(n1 k2) and does the 16-point DFT over n1 in
//           registers, which leaves it the 16 pixels k2 + 32 k1 (no swap);
// then the two q_z bins of those pixels are accumulated across z as in
// k_yz_tma.  The consumed input buffer is refilled (slice + 2) right after
// stage 1.  Waits are bounded as in k_col_fft4s_tma.  SEL: the z-first
// path's planes, as in k_yz_tma.
template <bool SEL>
__global__ void __launch_bounds__(512, 1) k_yz512_tma(const __grid_constant__ CUtensorMap tmap,
                                                      int nx, int nz, int nf, int ntiles, int L,
                                                      int T, const Geo<float>* __restrict__ geo,
                                                      const float2* __restrict__ twz_g,
                                                      const float2* __restrict__ twy_g,
                                                      const unsigned short* __restrict__ b0idx,
                                                      float4* __restrict__ part,
                                                      int* __restrict__ err, unsigned poll,
                                                      int kb, int zmask) {
  using C = float2;
  constexpr int TX = 16, NY = 512, TILE = NY * TX, STR = 33 * 8;
  constexpr unsigned kPoll = 1u << 22;
  extern __shared__ __align__(128) unsigned char smem_a128[];
  C* in = reinterpret_cast<C*>(smem_a128);  // [2][512][16], dense (TMA boxes)
  C* tr = in + 2 * TILE;                     // [32][STR]: (16 hw + k) x (n1 * 16 + col)
  C* twy = tr + 32 * STR;                    // [512]: W512^j
  C* twz = twy + NY;                         // [nz]
  unsigned short* btab = reinterpret_cast<unsigned short*>(twz + nz);  // [512][16]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(btab + TILE);
  const int t = threadIdx.x, w = t >> 5;
  const int col = t & 15;
  const int s0 = (int)blockIdx.x * L;
  const int s1 = s0 + L < T ? s0 + L : T;
  if (s0 >= s1) return;
  const long long npix = (long long)NY * nx;
  const int lognz = __ffs(nz) - 1;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async();
  }
  for (int i = t; i < NY; i += 512) twy[i] = twy_g[i];
  if constexpr (!SEL)
    for (int i = t; i < nz; i += 512) twz[i] = twz_g[i];
  __syncthreads();
  // step st -> (work item, slice or plane z)
  auto split = [&](int st, int& item, int& z) {
    if constexpr (SEL) {
      item = st / nz;
      z = st - item * nz;
    } else {
      item = st >> lognz;
      z = st & (nz - 1);
    }
  };
  auto issue = [&](int st, int b) {
    int item, z;
    split(st, item, z);
    const int f = item / ntiles, ti = item - f * ntiles;
    mbar_expect_tx(&bar[b], TILE * sizeof(C));
#pragma unroll
    for (int k = 0; k < 2; ++k)
      tma_load_3d(in + b * TILE + k * 256 * TX, &tmap, ti * 2 * TX, k * 256, f * nz + z, &bar[b]);
  };
  if (t == 0) {
    issue(s0, 0);
    if (s0 + 1 < s1) issue(s0 + 1, 1);
  }
  C acc0[16], acc1[16];
  int i = 0;
  for (int st = s0; st < s1; ++st, ++i) {
    const int b = i & 1;
    int item, z;
    split(st, item, z);
    const int ti = item % ntiles;
    if (z == 0 || st == s0) {  // a new segment: this tile's bins, zero accumulators
      __syncthreads();  // the previous step's reads of the bins are done
      for (int e = t; e < TILE; e += 512) {
        const int bin = b0idx[(size_t)(e >> 4) * nx + ti * TX + (e & 15)];
        btab[e] = (unsigned short)(SEL ? (bin - kb) & zmask : bin);
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) acc0[k] = acc1[k] = make_float2(0.f, 0.f);
    }
    const bool ok = mbar_wait_bounded(&bar[b], (i >> 1) & 1, poll);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicOr(err, 1);
        for (int d = 0; d < 2; ++d)
          if (st + d < s1) mbar_wait_bounded(&bar[(i + d) & 1], ((i + d) >> 1) & 1, kPoll);
      }
      return;
    }
    // stage 1: 16-point DFT of the samples n2 = 2m + hw of row n1
    {
      const int hw = w >> 3, n1 = (t >> 4) & 15;
      const C* src = in + b * TILE;
      C v[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) v[m] = src[(n1 + 16 * hw + 32 * m) * TX + col];
      dft_reg<16>(v);
      if (hw) w32_outputs<0>(v);
#pragma unroll
      for (int k = 0; k < 16; ++k) tr[(16 * hw + k) * STR + n1 * TX + col] = v[out_pos<16>(k)];
    }
    __syncthreads();  // stage-1 halves in tr, bins in place; the input buffer consumed
    if (t == 0 && st + 2 < s1) {
      fence_proxy_async();
      issue(st + 2, b);
    }
    // stage 2: X1[n1][k2] = E +- O' (minus for k2 >= 16), times W512^(n1 k2),
    // then the 16-point DFT over n1: pixels k2 + 32 k1
    {
      const int k2 = t >> 4, k = k2 & 15;
      const float sg = k2 >= 16 ? -1.f : 1.f;  // warp-uniform
      C v[16];
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) {
        const C e = tr[k * STR + n1 * TX + col];
        const C o = tr[(16 + k) * STR + n1 * TX + col];
        v[n1] = cmul(make_float2(fmaf(sg, o.x, e.x), fmaf(sg, o.y, e.y)), twy[n1 * k2]);
      }
      dft_reg<16>(v);
      const C wz = SEL ? make_float2(1.f, 0.f) : twz[z];
      float2* sel0 = nullptr;  // SEL: slot 0 of this thread's pixel column, as float2 pairs
      if constexpr (SEL)
        sel0 = reinterpret_cast<float2*>(part + (size_t)(item / ntiles) * npix + (size_t)ti * TX + col);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) {
        const int row = k2 + 32 * k1;
        const int b0 = btab[row * TX + col];
        if constexpr (SEL) {
          // each pixel's bins come from one plane each: stored as they pass
          float2* d = sel0 + 2 * (size_t)row * nx;
          if (b0 == z) d[0] = v[out_pos<16>(k1)];
          if (b0 + 1 == z) d[1] = v[out_pos<16>(k1)];
        } else {
          const C qq = cmul(v[out_pos<16>(k1)], twz[(b0 * z) & (nz - 1)]);
          acc0[k1] = cadd(acc0[k1], qq);
          acc1[k1] = cadd(acc1[k1], cmul(qq, wz));
        }
      }
      if (!SEL && (z == nz - 1 || st == s1 - 1)) {  // segment end: slot 0 if it began at z = 0
        // slot: this segment's place among the item's segments (0 if it
        // began at z = 0); L >= nz / 3 keeps it below kYzSlots
        const int item_start = st - z;
        const int slot = item_start >= s0 ? 0 : s0 / L - item_start / L;
        const int f = item / ntiles;
        float4* dst = part + ((size_t)slot * nf + f) * npix + (size_t)ti * TX + col;
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
          const int row = k2 + 32 * k1;
          dst[(size_t)row * nx] = make_float4(acc0[k1].x, acc0[k1].y, acc1[k1].x, acc1[k1].y);
        }
      }
    }
    __syncthreads();  // tr is rewritten by the next step
  }
}

// Eqs. (3Dscatter)/(Ewald) from the bins of k_yz_tma: per pixel, the two
// q_z bins of the three fields (slots 1-3 added where the item was split), the
// constant part returned at q = 0, the projection and the interpolation;
// written in fftshift order.
__global__ void k_ewald_bins(const float4* __restrict__ part, int nx, int ny, int nz,
                             int ntiles, int L, const Geo<float>* __restrict__ geo,
                             float dc0, float dc1, float dc2, float* __restrict__ img) {
  using C = float2;
  const long long npix = (long long)nx * ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const Geo<float> g = geo[pix];
  const int mx = (int)(pix % nx);
  float* dst = img + shifted_pixel(pix, nx, ny);
  if (g.b0 < 0) {
    *dst = 0.f;
    return;
  }
  const int ti = mx >> 3;
  C a0[3], a1[3];
  const float dcs[3] = {dc0, dc1, dc2};
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    float4 v = part[(size_t)f * npix + pix];
    // the 16-column work item; its segments (one per block it met)
    const int item = f * (ntiles >> 1) + (ti >> 1);
    const int nseg = ((item + 1) * nz - 1) / L - (item * nz) / L + 1;
    for (int sl = 1; sl < nseg; ++sl) {
      const float4 u = part[(size_t)(sl * 3 + f) * npix + pix];
      v.x += u.x; v.y += u.y; v.z += u.z; v.w += u.w;
    }
    a0[f] = make_float2(v.x, v.y);
    a1[f] = make_float2(v.z, v.w);
    if (pix == 0) {
      if (g.b0 == 0) a0[f].x += dcs[f];
      if (g.b1 == 0) a1[f].x += dcs[f];
    }
  }
  *dst = ewald_value<float>(g, a0, a1);
}

// Hot path, pipelined: a CTA owns PX consecutive pixels and streams their
// x/y-transformed slices P(z) through an S-stage ring in shared memory.  For
// each slice, thread 0 posts the byte count on the stage's mbarrier and
// issues three 1-D bulk copies (one per component, PX complex each); all
// threads wait on the barrier's phase, accumulate the two q_z bins of their
// two pixels from shared memory, synchronise, and the stage is refilled with
// slice z + S.  Every wait is bounded: on a timeout the CTA records the
// error in *err, waits (bounded) for its copies in flight, and returns.
template <typename R, int PX, int S>
__global__ void __launch_bounds__(PX / 2) k_ewald_tma(const typename RT<R>::C* __restrict__ p,
                                                      int nx, int ny, int nz,
                                                      const Geo<R>* __restrict__ geo,
                                                      const typename RT<R>::C* __restrict__ twz_g,
                                                      R dc0, R dc1, R dc2, R* __restrict__ img,
                                                      int* __restrict__ err, unsigned poll) {
  using C = typename RT<R>::C;
  constexpr unsigned kPoll = 1u << 22;
  constexpr unsigned kBytes = PX * sizeof(C);
  extern __shared__ __align__(128) unsigned char smem_a128[];
  C* stage = reinterpret_cast<C*>(smem_a128);                       // [S][3][PX]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(stage + S * 3 * PX);
  C* twz = reinterpret_cast<C*>(bar + S);                           // [nz]
  const long long npix = (long long)nx * ny;
  const size_t N = (size_t)npix * nz;
  const long long pix_base = (long long)blockIdx.x * PX;
  const C* src = p + pix_base;
  const int t = threadIdx.x;

  if (t == 0) {
    for (int st = 0; st < S; ++st) mbar_init(&bar[st], 1);
    fence_proxy_async();
  }
  for (int i = t; i < nz; i += PX / 2) twz[i] = twz_g[i];
  __syncthreads();
  auto issue = [&](int z, int st) {
    mbar_expect_tx(&bar[st], 3 * kBytes);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      bulk_g2s(stage + (st * 3 + k) * PX, src + k * N + (size_t)z * npix, kBytes, &bar[st]);
  };
  if (t == 0)
    for (int z = 0; z < S && z < nz; ++z) issue(z, z);

  const long long pix0 = pix_base + 2 * t;
  Geo<R> g[2];
  g[0] = geo[pix0];
  g[1] = geo[pix0 + 1];
  const int s0[2] = {g[0].b0 < 0 ? 0 : g[0].b0, g[1].b0 < 0 ? 0 : g[1].b0};
  const int s1[2] = {g[0].b1 < 0 ? 0 : g[0].b1, g[1].b1 < 0 ? 0 : g[1].b1};
  int i0[2] = {0, 0}, i1[2] = {0, 0};
  C a0[2][3], a1[2][3];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < 3; ++k) a0[q][k] = a1[q][k] = RT<R>::mk(0, 0);

  int failed_at = -1;
  for (int z = 0; z < nz; ++z) {
    const int st = z % S;
    const bool ok = mbar_wait_bounded(&bar[st], (z / S) & 1, poll);
    if (__syncthreads_or(!ok)) {
      failed_at = z;
      break;
    }
    const C* sp = stage + st * 3 * PX + 2 * t;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const C v0 = sp[k * PX], v1 = sp[k * PX + 1];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const C v = q ? v1 : v0;
        a0[q][k] = cadd(a0[q][k], cmul(v, twz[i0[q]]));
        a1[q][k] = cadd(a1[q][k], cmul(v, twz[i1[q]]));
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      i0[q] += s0[q];
      if (i0[q] >= nz) i0[q] -= nz;
      i1[q] += s1[q];
      if (i1[q] >= nz) i1[q] -= nz;
    }
    __syncthreads();  // every thread is done with this stage
    if (t == 0 && z + S < nz) {
      fence_proxy_async();
      issue(z + S, st);
    }
  }
  if (failed_at >= 0) {
    if (t == 0) {
      atomicOr(err, 1);
      // slices failed_at .. failed_at + S - 1 were issued and not consumed:
      // let their copies land (bounded) before the CTA's shared memory goes
      for (int z = failed_at; z < nz && z < failed_at + S; ++z)
        mbar_wait_bounded(&bar[z % S], (z / S) & 1, kPoll);
    }
    return;
  }
  if (pix0 == 0) {
    const R dcs[3] = {dc0, dc1, dc2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (g[0].b0 == 0) a0[0][k].x += dcs[k];
      if (g[0].b1 == 0) a1[0][k].x += dcs[k];
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const long long pix = pix0 + q;
    img[shifted_pixel(pix, nx, ny)] = g[q].b0 < 0 ? R(0) : ewald_value<R>(g[q], a0[q], a1[q]);
  }
}

// One thread per pixel with plain loads: the pruned z transform for grids
// with an odd pixel count (where pixel pairs are not 16-byte aligned).
template <typename R>
__global__ void __launch_bounds__(256) k_ewald_each(const typename RT<R>::C* __restrict__ p,
                                                    int nx, int ny, int nz,
                                                    const Geo<R>* __restrict__ geo,
                                                    const typename RT<R>::C* __restrict__ twz,
                                                    R dc0, R dc1, R dc2, R* __restrict__ img) {
  using C = typename RT<R>::C;
  const long long npix = (long long)nx * ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const Geo<R> g = geo[pix];
  R* dst = img + shifted_pixel(pix, nx, ny);
  if (g.b0 < 0) {
    *dst = R(0);
    return;
  }
  const size_t N = (size_t)npix * nz;
  C a0[3], a1[3];
  for (int k = 0; k < 3; ++k) a0[k] = a1[k] = RT<R>::mk(0, 0);
  int i0 = 0, i1 = 0;
  for (int z = 0; z < nz; ++z) {
    for (int k = 0; k < 3; ++k) {
      const C v = p[k * N + (size_t)z * npix + pix];
      a0[k] = cadd(a0[k], cmul(v, twz[i0]));
      a1[k] = cadd(a1[k], cmul(v, twz[i1]));
    }
    i0 += g.b0;
    if (i0 >= nz) i0 -= nz;
    i1 += g.b1;
    if (i1 >= nz) i1 -= nz;
  }
  if (pix == 0) {
    const R dcs[3] = {dc0, dc1, dc2};
    for (int k = 0; k < 3; ++k) {
      if (g.b0 == 0) a0[k].x += dcs[k];
      if (g.b1 == 0) a1[k].x += dcs[k];
    }
  }
  *dst = ewald_value<R>(g, a0, a1);
}

// ------------------------------------------------ linearity fast path
// p~(alpha) = cos(alpha) F(N_t x) + sin(alpha) F(N_t y): the five FFT'd
// N_t entries are reduced once per energy to the two q_z bins each pixel
// needs (k_zbins5); each angle then only combines them per pixel
// (k_ewald_linear).
template <typename R, int ZB>
__global__ void __launch_bounds__(256) k_zbins5(const typename RT<R>::C* __restrict__ f, int nx, int ny,
                                                int nz, const Geo<R>* __restrict__ geo,
                                                const typename RT<R>::C* __restrict__ twz_g,
                                                int tw_in_smem, R dc,
                                                typename RT<R>::C* __restrict__ bins) {
  using C = typename RT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tws = reinterpret_cast<C*>(smem_raw);
  if (tw_in_smem) {
    for (int i = threadIdx.x; i < nz; i += blockDim.x) tws[i] = twz_g[i];
    __syncthreads();
  }
  const C* twz = tw_in_smem ? tws : twz_g;
  const long long npix = (long long)nx * ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const size_t N = (size_t)npix * nz;
  const Geo<R> g = geo[pix];
  const int s0 = g.b0 < 0 ? 0 : g.b0, s1 = g.b1 < 0 ? 0 : g.b1;
  C a0[5], a1[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) a0[q] = a1[q] = RT<R>::mk(0, 0);
  int i0 = 0, i1 = 0;
  const C* src = f + pix;
  int z = 0;
  if (g.b0 >= 0) {
    for (; z + ZB <= nz; z += ZB) {
      C v[ZB][5];
#pragma unroll
      for (int u = 0; u < ZB; ++u)
#pragma unroll
        for (int q = 0; q < 5; ++q) v[u][q] = __ldg(src + q * N + (size_t)(z + u) * npix);
#pragma unroll
      for (int u = 0; u < ZB; ++u) {
        const C w0 = twz[i0], w1 = twz[i1];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          a0[q] = cadd(a0[q], cmul(v[u][q], w0));
          a1[q] = cadd(a1[q], cmul(v[u][q], w1));
        }
        i0 += s0;
        if (i0 >= nz) i0 -= nz;
        i1 += s1;
        if (i1 >= nz) i1 -= nz;
      }
    }
    for (; z < nz; ++z) {
      const C w0 = twz[i0], w1 = twz[i1];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const C v = __ldg(src + q * N + (size_t)z * npix);
        a0[q] = cadd(a0[q], cmul(v, w0));
        a1[q] = cadd(a1[q], cmul(v, w1));
      }
      i0 += s0;
      if (i0 >= nz) i0 -= nz;
      i1 += s1;
      if (i1 >= nz) i1 -= nz;
    }
    if (pix == 0) {  // diagonal entries xx (0) and yy (2) get the constant back
      if (g.b0 == 0) { a0[0].x += dc; a0[2].x += dc; }
      if (g.b1 == 0) { a1[0].x += dc; a1[2].x += dc; }
    }
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    bins[(size_t)(2 * q) * npix + pix] = a0[q];
    bins[(size_t)(2 * q + 1) * npix + pix] = a1[q];
  }
}

// The linearity path's per-energy bins from the fused y+z pass over the
// five FFT'd N_t entries (k_yz_tma with five fields): slots added, the
// constant returned to xx and yy at q = 0, and the k_zbins5 layout written
// (bins[2q] = bin b0, bins[2q + 1] = bin b0 + 1 of entry q; zero off the
// sphere).
__global__ void __launch_bounds__(256) k_bins5_from_part(const float4* __restrict__ part, int nx,
                                                         int ny, int nz, int ntiles, int L,
                                                         const Geo<float>* __restrict__ geo,
                                                         float dc, float2* __restrict__ bins) {
  const long long npix = (long long)nx * ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const Geo<float> g = geo[pix];
  const int ti = (int)(pix % nx) >> 3;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (g.b0 >= 0) {
      v = part[(size_t)q * npix + pix];
      const int item = q * (ntiles >> 1) + (ti >> 1);
      const int nseg = ((item + 1) * nz - 1) / L - (item * nz) / L + 1;
      for (int sl = 1; sl < nseg; ++sl) {
        const float4 u = part[(size_t)(sl * 5 + q) * npix + pix];
        v.x += u.x; v.y += u.y; v.z += u.z; v.w += u.w;
      }
      if (pix == 0 && (q == 0 || q == 2)) {
        if (g.b0 == 0) v.x += dc;
        if (g.b1 == 0) v.z += dc;
      }
    }
    bins[(size_t)(2 * q) * npix + pix] = make_float2(v.x, v.y);
    bins[(size_t)(2 * q + 1) * npix + pix] = make_float2(v.z, v.w);
  }
}

// Detector value of one pixel for e = (ce, se, 0) from the linearity
// bins (Eq. (Ewald) with p~ = N_t~ e per bin; zero off the sphere).
template <typename R>
__device__ __forceinline__ R linear_pixel(const typename RT<R>::C* __restrict__ bins, long long npix,
                                          long long pix, const Geo<R>& g, R ce, R se,
                                          int literal) {
  using C = typename RT<R>::C;
  if (g.b0 < 0) return R(0);
  C pb[2][3];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    C t[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) t[q] = bins[(size_t)(2 * q + b) * npix + pix];
    // columns x = (xx, xy, xz) and y = (xy, yy, yz) of N_t, combined with e
    const C px = RT<R>::mk(ce * t[0].x + se * t[1].x, ce * t[0].y + se * t[1].y);
    const C py = RT<R>::mk(ce * t[1].x + se * t[2].x, ce * t[1].y + se * t[2].y);
    const C pz = RT<R>::mk(ce * t[3].x + se * t[4].x, ce * t[3].y + se * t[4].y);
    if (literal) {
      pb[b][0] = RT<R>::mk(ce * px.x + se * py.x, ce * px.y + se * py.y);
      pb[b][1] = RT<R>::mk(-se * px.x + ce * py.x, -se * px.y + ce * py.y);
    } else {
      pb[b][0] = px;
      pb[b][1] = py;
    }
    pb[b][2] = pz;
  }
  return ewald_value<R>(g, pb[0], pb[1]);
}

template <typename R>
__global__ void __launch_bounds__(256) k_ewald_linear(const typename RT<R>::C* __restrict__ bins, int nx,
                                                      int ny, const Geo<R>* __restrict__ geo, R ce,
                                                      R se, int literal, R* __restrict__ img) {
  const long long npix = (long long)nx * ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  img[shifted_pixel(pix, nx, ny)] = linear_pixel<R>(bins, npix, pix, geo[pix], ce, se, literal);
}

// The same for a batch of angles: imgs[a] for a = blockIdx.y.
template <typename R>
__global__ void __launch_bounds__(256) k_ewald_linear_many(const typename RT<R>::C* __restrict__ bins,
                                                           int nx, int ny,
                                                           const Geo<R>* __restrict__ geo,
                                                           AngleBatch<R> ab, int literal,
                                                           R* __restrict__ imgs) {
  const long long npix = (long long)nx * ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const int a = blockIdx.y;
  imgs[(size_t)a * npix + shifted_pixel(pix, nx, ny)] =
      linear_pixel<R>(bins, npix, pix, geo[pix], ab.ce[a], ab.se[a], literal);
}

// ------------------------------------------------ Algorithm 3 (NrComputation)
// N_t = sum_j (N_rot^j N_rot^j - I) / (4 pi) with N_rot^2 - I =
// (a^2 - 1) I + (2ab + b^2) d d^T, stored as the five entries an in-plane e
// reads (xx, xy, yy, xz, yz; zz is never used), nt[5][N], with the
// constant -(c - 1)/(4 pi) removed from the diagonal as in Algorithm 1.
template <typename R> struct NtAcc {
  R aw;          // sum_j v_j^2
  R as[2];       // sum_j v_j^2 tau' (2 + tau')
  R g[5][2];     // sum_j (2ab + b^2) d d^T entries xx, xy, yy, xz, yz
};

template <typename R>
__device__ __forceinline__ void nt_add(NtAcc<R>& A, R v, R s, R phi, R theta,
                                       const PolParams<R>& pp, int j) {
  const R tpr = pp.tau[j][0] + s * pp.dperp[j][0];
  const R tpi = pp.tau[j][1] + s * pp.dperp[j][1];
  const R v2 = v * v;
  A.aw += v2;
  A.as[0] += v2 * (tpr * (R(2) + tpr) - tpi * tpi);
  A.as[1] += v2 * (tpi * (R(2) + tpr) + tpr * tpi);
  const R vs = v * s;
  const R br = vs * pp.dpar[j][0], bi = vs * pp.dpar[j][1];
  const R qr = R(2) * v * (R(1) + tpr) + br, qi = R(2) * v * tpi + bi;
  const R gr = br * qr - bi * qi, gi = br * qi + bi * qr;
  R sp, cp, st, ct;
  sincos_r(phi, &sp, &cp);
  sincos_r(theta, &st, &ct);
  const R dx = cp * st, dy = sp * st, dz = ct;
  const R dd[5] = {dx * dx, dx * dy, dy * dy, dx * dz, dy * dz};
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    A.g[q][0] += gr * dd[q];
    A.g[q][1] += gi * dd[q];
  }
}

// All components from device-resident M: one pass, N_t written once.
template <typename R>
__global__ void __launch_bounds__(256) k_nt_all(const typename RT<R>::V4* __restrict__ M, long long N,
                                                PolParams<R> pp, typename RT<R>::C* __restrict__ nt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  NtAcc<R> A = {};
  for (int j = 0; j < pp.c; ++j) {
    const typename RT<R>::V4 m = M[(size_t)j * N + i];
    nt_add(A, (R)m.x, (R)m.y, (R)m.z, (R)m.w, pp, j);
  }
  const R inv = R(1.0 / kFourPi);
  const R dr = (A.aw - R(1)) + A.as[0], di = A.as[1];
  const R diag[5] = {R(1), R(0), R(1), R(0), R(0)};
#pragma unroll
  for (int q = 0; q < 5; ++q)
    nt[q * (size_t)N + i] = RT<R>::mk((A.g[q][0] + diag[q] * dr) * inv, (A.g[q][1] + diag[q] * di) * inv);
}

// One component j over the voxel range [off, off + n) from a staging copy
// (Algorithm 3's per-material streaming).  FIRST writes, later components add.
template <typename R, bool FIRST>
__global__ void __launch_bounds__(256) k_nt_comp(const typename RT<R>::V4* __restrict__ Mj,
                                                 long long off, long long n, long long N, int j,
                                                 PolParams<R> pp, typename RT<R>::C* __restrict__ nt) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const size_t i = (size_t)(off + t);
  NtAcc<R> A = {};
  const typename RT<R>::V4 m = Mj[t];
  nt_add(A, (R)m.x, (R)m.y, (R)m.z, (R)m.w, pp, j);
  const R inv = R(1.0 / kFourPi);
  // the first component carries the -1 of (sum v^2 - 1)
  const R dr = (FIRST ? A.aw - R(1) : A.aw) + A.as[0], di = A.as[1];
  const R diag[5] = {R(1), R(0), R(1), R(0), R(0)};
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    typename RT<R>::C v =
        RT<R>::mk((A.g[q][0] + diag[q] * dr) * inv, (A.g[q][1] + diag[q] * di) * inv);
    if (!FIRST) v = cadd(v, nt[q * (size_t)N + i]);
    nt[q * (size_t)N + i] = v;
  }
}

// N_t for output: the removed constant restored on the diagonal.
template <typename R>
__global__ void k_nt_restore(const typename RT<R>::C* __restrict__ nt, typename RT<R>::C* __restrict__ out,
                             long long N, R ref) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 5 * N) return;
  typename RT<R>::C v = nt[i];
  const int q = (int)(i / N);
  if (q == 0 || q == 2) v.x += ref;
  out[i] = v;
}

// ------------------------------------------------------- detector rotation
// acc(Q) += img(U(alpha) Q), bilinear, zero outside; pixel coordinates in
// fftshift order with centre (nx/2, ny/2) and the q-spacing ratio nx/ny.
// One 16 x 16 tile of output pixels per CTA, so that the source footprint
// of a CTA is a compact rotated square.  The source position is computed in
// fixed point with 48 fractional bits: cos/sin (times the aspect ratio) are
// integers scaled by 2^48 and the offsets from the centre are integers, so
// the only error is the coefficients' rounding, 2^-49 of a pixel per pixel
// of offset (an FP64 evaluation errs by about 2^-52 |position|); every term
// stays below 2^60 for n <= 4096.  The floor is a shift and the fraction a
// mask (no FP64 arithmetic).
constexpr int kRotTile = 16;
// Bilinear sample of img (fftshift order) at U(alpha) Q for the output
// pixel (ix, iy); the coefficients are cos/sin (with the aspect ratios) in
// 2^-48 fixed point, so the source position is exact to 2^-49 pixel.
template <typename R>
__device__ __forceinline__ R rotated_sample(const R* __restrict__ img, int nx, int ny, int ix,
                                            int iy, long long cxx, long long cxy, long long cyx,
                                            long long cyy) {
  const int cx = nx / 2, cy = ny / 2;
  const long long dx = ix - cx, dy = iy - cy;
  const long long fx = ((long long)cx << 48) + cxx * dx - cxy * dy;
  const long long fy = ((long long)cy << 48) + cyx * dx + cyy * dy;
  const int x0 = (int)(fx >> 48), y0 = (int)(fy >> 48);
  const R scale = R(1.0 / 281474976710656.0);  // 2^-48
  const R tx = (R)(fx & ((1LL << 48) - 1)) * scale;
  const R ty = (R)(fy & ((1LL << 48) - 1)) * scale;
  R val = R(0);
#pragma unroll
  for (int dyy = 0; dyy < 2; ++dyy) {
    const int yy = y0 + dyy;
    if (yy < 0 || yy >= ny) continue;
    const R wy = dyy ? ty : R(1) - ty;
#pragma unroll
    for (int dxx = 0; dxx < 2; ++dxx) {
      const int xx = x0 + dxx;
      if (xx < 0 || xx >= nx) continue;
      const R wx = dxx ? tx : R(1) - tx;
      val += wy * wx * __ldg(img + (size_t)yy * nx + xx);
    }
  }
  return val;
}

template <typename R>
__global__ void __launch_bounds__(kRotTile * kRotTile) k_rotate_acc(const R* __restrict__ img,
                                                                    R* __restrict__ acc, int nx,
                                                                    int ny, long long cxx,
                                                                    long long cxy, long long cyx,
                                                                    long long cyy, int rotate) {
  const int ix = blockIdx.x * kRotTile + threadIdx.x;
  const int iy = blockIdx.y * kRotTile + threadIdx.y;
  if (ix >= nx || iy >= ny) return;
  const size_t pix = (size_t)iy * nx + ix;
  acc[pix] += rotate ? rotated_sample<R>(img, nx, ny, ix, iy, cxx, cxy, cyx, cyy) : img[pix];
}

// A batch of angles at once: acc += sample of imgs[0], then imgs[1], ...,
// in that order (the same sums as one k_rotate_acc launch per angle).
template <typename R>
__global__ void __launch_bounds__(kRotTile * kRotTile) k_rotate_acc_many(const R* __restrict__ imgs,
                                                                         R* __restrict__ acc,
                                                                         int nx, int ny,
                                                                         AngleBatch<R> ab,
                                                                         int rotate) {
  const int ix = blockIdx.x * kRotTile + threadIdx.x;
  const int iy = blockIdx.y * kRotTile + threadIdx.y;
  if (ix >= nx || iy >= ny) return;
  const size_t npix = (size_t)nx * ny, pix = (size_t)iy * nx + ix;
  R sum = acc[pix];
  for (int a = 0; a < ab.n; ++a) {
    const R* img = imgs + (size_t)a * npix;
    sum += rotate ? rotated_sample<R>(img, nx, ny, ix, iy, ab.cxx[a], ab.cxy[a], ab.cyx[a],
                                      ab.cyy[a])
                  : img[pix];
  }
  acc[pix] = sum;
}

template <typename R>
__global__ void k_scale(const R* __restrict__ acc, R* __restrict__ out, long long n, R scale) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = acc[i] * scale;
}

// Sec. 3.1 ranges: 0 <= v <= 1, 0 <= s <= 1, finite angles.  Sets *flag.
template <typename R>
__global__ void k_validate(const R* __restrict__ M, long long n_entries, int* __restrict__ flag) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_entries) return;
  const R v = M[4 * i], s = M[4 * i + 1], ph = M[4 * i + 2], th = M[4 * i + 3];
  const bool ok = (v >= R(0)) && (v <= R(1)) && (s >= R(0)) && (s <= R(1)) && isfinite(ph) &&
                  isfinite(th);
  if (!ok) atomicOr(flag, 1);
}

// The director d = (cos phi sin theta, sin phi sin theta, cos theta) of
// every component and voxel (Eq. (rotBCD)), dir[j][3][N]: it depends on the
// morphology alone, so FP64 runs evaluate its sines and cosines once per
// morphology rather than once per voxel, component, energy and angle.
template <typename R>
__global__ void k_director(const typename RT<R>::V4* __restrict__ M, long long n_entries,
                           long long N, R* __restrict__ dir) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_entries) return;
  const typename RT<R>::V4 m = M[i];
  R sp, cp, st, ct;
  sincos_r((R)m.z, &sp, &cp);
  sincos_r((R)m.w, &st, &ct);
  const long long j = i / N, v = i - j * N;
  R* d = dir + (size_t)j * 3 * N + v;
  d[0] = cp * st;
  d[N] = sp * st;
  d[2 * N] = ct;
}

// ================================================================ launchers
static inline int ilog2(long long n) {
  int l = 0;
  while ((1LL << l) < n) ++l;
  return l;
}
static inline unsigned grid1(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename R, int T, int EC, bool DO_FFT, int LOGNX, bool FROM_NT>
static cudaError_t pol_fftx_impl(const void* M, int nx, int ny, int nz, const PolParams<R>& pp,
                                 void* p, const void* twx, const void* nt, long long row_begin,
                                 long long row_count, cudaStream_t s, const void* dir) {
  using C = typename RT<R>::C;
  const long long N = (long long)nx * ny * nz;
  // Without the FFT the voxels are independent: treat them as N rows of one.
  const int lognx = DO_FFT ? ilog2(nx) : 0;
  long long nrows = DO_FFT ? (long long)ny * nz : N;
  if (DO_FFT && row_count >= 0) nrows = row_count;
  else row_begin = 0;
  const int rows = DO_FFT ? EC / nx : EC;
  size_t smem = DO_FFT ? padded(3 * EC) * sizeof(C) : 0;
  int tw_in_smem = 0;
  if (DO_FFT && smem + nx * sizeof(C) <= 200 * 1024) {
    smem += nx * sizeof(C);
    tw_in_smem = 1;
  }
  auto kern = k_pol_fftx<R, T, EC, DO_FFT, LOGNX, FROM_NT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (nrows <= 0) return cudaSuccess;
  kern<<<grid1(nrows, rows), T, smem, s>>>((const typename RT<R>::V4*)M, N, lognx, row_begin,
                                           row_begin + nrows, pp, (C*)p, (const C*)twx,
                                           tw_in_smem, (const C*)nt, (const R*)dir);
  return cudaGetLastError();
}

template <typename R, bool FROM_NT>
static cudaError_t pol_fftx_dispatch(const void* M, int nx, int ny, int nz, const PolParams<R>& pp,
                                     bool do_fft, void* p, const void* twx, const void* nt,
                                     long long rb, long long rc, cudaStream_t s, const void* dir) {
  if (!do_fft)
    return pol_fftx_impl<R, 256, 1024, false, -1, FROM_NT>(M, nx, ny, nz, pp, p, twx, nt, rb, rc, s,
                                                           dir);
  if (nx & (nx - 1)) {
    // other lengths: polarisation alone, then the mixed-radix x-FFT of the
    // 3 ny nz rows in place
    if (rc >= 0) return cudaErrorInvalidValue;
    cudaError_t e = pol_fftx_impl<R, 256, 1024, false, -1, FROM_NT>(M, nx, ny, nz, pp, p, twx, nt,
                                                                    0, -1, s, dir);
    if (e != cudaSuccess) return e;
    return launch_row_fft<R>(p, nx, 3LL * ny * nz, twx, s);
  }
#define RSX_POL(L)                                                                          \
  case L:                                                                                   \
    return pol_fftx_impl<R, 256, 1024, true, L, FROM_NT>(M, nx, ny, nz, pp, p, twx, nt, rb, rc, \
                                                         s, dir);
  switch (ilog2(nx)) {
    RSX_POL(6) RSX_POL(7) RSX_POL(8) RSX_POL(9) RSX_POL(10)
    case 11:
      return pol_fftx_impl<R, 256, 2048, true, 11, FROM_NT>(M, nx, ny, nz, pp, p, twx, nt, rb, rc,
                                                            s, dir);
    case 12:
      return pol_fftx_impl<R, 512, 4096, true, 12, FROM_NT>(M, nx, ny, nz, pp, p, twx, nt, rb, rc,
                                                            s, dir);
    default:
      return pol_fftx_impl<R, 256, 1024, true, -1, FROM_NT>(M, nx, ny, nz, pp, p, twx, nt, rb, rc,
                                                            s, dir);
  }
#undef RSX_POL
}

template <typename R>
cudaError_t launch_pol_fftx(const void* M, int nx, int ny, int nz, const PolParams<R>& pp,
                            bool do_fft, void* p, const void* twx, cudaStream_t s,
                            long long row_begin, long long row_count, const void* dir) {
  return pol_fftx_dispatch<R, false>(M, nx, ny, nz, pp, do_fft, p, twx, nullptr, row_begin,
                                     row_count, s, dir);
}

template <typename R>
cudaError_t launch_ntp_fftx(const void* nt, int nx, int ny, int nz, const PolParams<R>& pp,
                            bool do_fft, void* p, const void* twx, cudaStream_t s,
                            long long row_begin, long long row_count) {
  return pol_fftx_dispatch<R, true>(nullptr, nx, ny, nz, pp, do_fft, p, twx, nt, row_begin,
                                    row_count, s, nullptr);
}

template <typename R>
cudaError_t launch_director(const void* M, long long n_entries, long long N, void* dir,
                            cudaStream_t s) {
  if (n_entries == 0) return cudaSuccess;
  k_director<R><<<grid1(n_entries, 256), 256, 0, s>>>((const typename RT<R>::V4*)M, n_entries, N,
                                                      (R*)dir);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pol_fft4s(const void* M, const void* nt, int nx, int ny, int nz,
                             const PolParams<R>& pp, void* p, const void* tw4, cudaStream_t s,
                             const void* dir) {
  using C = typename RT<R>::C;
  if (nx != 1024) return cudaErrorInvalidValue;
  const long long N = (long long)nx * ny * nz, nrows = (long long)ny * nz;
  const size_t smem = (3 * 32 * 33 + 1024) * sizeof(C);
  if (nt) {
    auto kern = k_pol_fft4s<R, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nrows, 128, smem, s>>>(nullptr, N, nrows, pp, (C*)p, (const C*)tw4,
                                            (const C*)nt, nullptr);
  } else {
    auto kern = k_pol_fft4s<R, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nrows, 128, smem, s>>>((const typename RT<R>::V4*)M, N, nrows, pp, (C*)p,
                                            (const C*)tw4, nullptr, (const R*)dir);
  }
  return cudaGetLastError();
}

template <bool NT, int NX>
static cudaError_t pol_fft4s_tma_impl(const void* src, int nx, int ny, int nz,
                                      const PolParams<float>& pp, void* p, const void* tw4, int* err,
                                      int n_sm, unsigned poll, cudaStream_t s) {
  // 2 row buffers, 4 polarisation warps, one transform group, 48 KB of
  // stages (rows of morphology components or of N_t entries): ~106 KB of
  // shared memory for 1024-point rows, ~78 KB for 512, 256 threads, two
  // blocks per SM
  constexpr size_t elem = NT ? sizeof(float2) : sizeof(float4);
  constexpr int S = (int)(48 * 1024 / (NX * elem)), NP = 2, PW = 4, FG = 1, CPS = 2;
  if (nx != NX || n_sm <= 0 || ((uintptr_t)src & 15)) return cudaErrorInvalidValue;
  const long long N = (long long)nx * ny * nz, nrows = (long long)ny * nz;
  if (nrows <= 0) return cudaSuccess;
  const size_t smem = (size_t)S * NX * elem + (NP * 3 * (NX / 32) * 33 + 1024) * sizeof(float2) +
                      2 * S * 8 + 16;
  auto kern = k_pol_fft4s_tma<S, NP, PW, FG, NT, NX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  const long long grid = nrows < (long long)CPS * n_sm ? nrows : (long long)CPS * n_sm;
  kern<<<(unsigned)grid, 32 * (PW + 3 * FG + 1), smem, s>>>(src, N, nrows, pp, (float2*)p,
                                                            (const float2*)tw4, err, poll);
  return cudaGetLastError();
}

cudaError_t launch_pol_fft4s_tma(const void* M, int nx, int ny, int nz, const PolParams<float>& pp,
                                 void* p, const void* tw, int* err, int n_sm, unsigned poll,
                                 cudaStream_t s) {
  return nx == 512 ? pol_fft4s_tma_impl<false, 512>(M, nx, ny, nz, pp, p, tw, err, n_sm, poll, s)
                   : pol_fft4s_tma_impl<false, 1024>(M, nx, ny, nz, pp, p, tw, err, n_sm, poll, s);
}

cudaError_t launch_ntp_fft4s_tma(const void* nt, int nx, int ny, int nz,
                                 const PolParams<float>& pp, void* p, const void* tw, int* err,
                                 int n_sm, unsigned poll, cudaStream_t s) {
  return nx == 512 ? pol_fft4s_tma_impl<true, 512>(nt, nx, ny, nz, pp, p, tw, err, n_sm, poll, s)
                   : pol_fft4s_tma_impl<true, 1024>(nt, nx, ny, nz, pp, p, tw, err, n_sm, poll, s);
}

template <int NX>
static cudaError_t pol_fft4s_tma_multi_impl(const void* M, int ny, int nz,
                                            const PolParams<float>& pp, const XAngles& ang,
                                            void* p, long long pstride, const void* tw,
                                            int* err, int n_sm, unsigned poll, cudaStream_t s) {
  // 512- and 1024-point rows: 3 stages of one (row, component) slice, 6 row
  // buffers, 8 polarisation warps (NX / 256 voxels per thread), three
  // transform groups (the transforms are the larger share of the work; a
  // fourth would cut the registers below what a transform needs) and a
  // producer warp: one 576-thread block per SM, ~205 KB of shared memory
  // for 1024-point rows.  2048-point rows: 1024-voxel segments, 3 row
  // buffers of 50 KB (so at most 3 angles per launch), ~213 KB.
  constexpr int S = 3, NPB = NX == 2048 ? 3 : 6, PW = 8, FG = 3;
  constexpr int FS = NX == 2048 ? 2 * 1056 : (NX / 32) * 33;
  constexpr int SV = NX > 1024 ? 1024 : NX, NTW = NX == 2048 ? 2048 : 1024;
  if (n_sm <= 0 || ((uintptr_t)M & 15) || ang.n < 1 || ang.n > 8 ||
      (NX == 2048 && ang.n > NPB))
    return cudaErrorInvalidValue;
  const long long N = (long long)NX * ny * nz, nrows = (long long)ny * nz;
  if (nrows <= 0) return cudaSuccess;
  const size_t smem = (size_t)S * SV * sizeof(float4) + ((size_t)NPB * 3 * FS + NTW) * sizeof(float2) +
                      2 * S * 8 + 16;
  auto kern = k_pol_fft4s_tma_multi<S, NPB, PW, FG, NX, 8>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  const long long grid = nrows < (long long)n_sm ? nrows : (long long)n_sm;
  kern<<<(unsigned)grid, 32 * (PW + 3 * FG + 1), smem, s>>>(
      (const float4*)M, N, nrows, pp, ang, (float2*)p, pstride, (const float2*)tw, err, poll);
  return cudaGetLastError();
}

cudaError_t launch_pol_fft4s_tma_multi(const void* M, int nx, int ny, int nz,
                                       const PolParams<float>& pp, const XAngles& ang, void* p,
                                       long long pstride, const void* tw, int* err, int n_sm,
                                       unsigned poll, cudaStream_t s) {
  if (nx == 1024)
    return pol_fft4s_tma_multi_impl<1024>(M, ny, nz, pp, ang, p, pstride, tw, err, n_sm, poll, s);
  if (nx == 512)
    return pol_fft4s_tma_multi_impl<512>(M, ny, nz, pp, ang, p, pstride, tw, err, n_sm, poll, s);
  if (nx == 2048)
    return pol_fft4s_tma_multi_impl<2048>(M, ny, nz, pp, ang, p, pstride, tw, err, n_sm, poll, s);
  return cudaErrorInvalidValue;
}

template <int R>
static cudaError_t pol_zfft_impl(const void* tmap, int nx, int ny, const PolParams<float>& pp,
                                 const XAngles& ang, void* out, long long kstride,
                                 long long fstride, int kb, int ns, const void* twz, int* err,
                                 int n_sm, unsigned poll, cudaStream_t s) {
  // as the multi-angle x pass: 3 stages (one component of a 1024-voxel
  // tile each), 6 row buffers, 8 polarisation warps, three transform groups
  // and a producer: one 576-thread block per SM, ~200 KB of shared memory
  // for nz = 128
  constexpr int S = 3, NPB = 6, PW = 8, FG = 3;
  using Lay = ZfLayout<R>;
  if (n_sm <= 0 || ang.n < 1 || ang.n > kMaxXAngles || nx % Lay::XW || ns < 1 || ns > Lay::NZ ||
      kb < 0 || kb >= Lay::NZ)
    return cudaErrorInvalidValue;
  const long long npix = (long long)nx * ny, ntiles = npix / Lay::XW;
  if (ntiles <= 0) return cudaSuccess;
  const size_t smem = (size_t)S * 1024 * sizeof(float4) +
                      ((size_t)NPB * 3 * Lay::FS + 32 * R) * sizeof(float2) + 2 * S * 8 + 16;
  auto kern = k_pol_zfft_multi<R, S, NPB, PW, FG, kMaxXAngles>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  const long long grid = ntiles < (long long)n_sm ? ntiles : (long long)n_sm;
  kern<<<(unsigned)grid, 32 * (PW + 3 * FG + 1), smem, s>>>(
      *(const CUtensorMap*)tmap, nx, npix, ntiles, pp, ang, (float2*)out, kstride, fstride, kb, ns,
      (const float2*)twz, err, poll);
  return cudaGetLastError();
}

bool zfirst_fusable(int nx, int ny, int nz) {
  return (nz == 32 || nz == 64 || nz == 128) && (nx == 512 || nx == 1024 || nx == 2048) &&
         (ny == 512 || ny == 1024 || ny == 2048);
}

cudaError_t launch_pol_zfft_multi(const void* tmap, int nx, int ny, int nz,
                                  const PolParams<float>& pp, const XAngles& ang, void* out,
                                  long long kstride, long long fstride, int kb, int ns,
                                  const void* twz, int* err, int n_sm, unsigned poll,
                                  cudaStream_t s) {
  if (!zfirst_fusable(nx, ny, nz)) return cudaErrorInvalidValue;
  if (nz == 128)
    return pol_zfft_impl<4>(tmap, nx, ny, pp, ang, out, kstride, fstride, kb, ns, twz, err, n_sm,
                            poll, s);
  if (nz == 64)
    return pol_zfft_impl<2>(tmap, nx, ny, pp, ang, out, kstride, fstride, kb, ns, twz, err, n_sm,
                            poll, s);
  return pol_zfft_impl<1>(tmap, nx, ny, pp, ang, out, kstride, fstride, kb, ns, twz, err, n_sm,
                          poll, s);
}

template <int NX, int W>
static cudaError_t xfft_rows_impl(void* data, long long nrows, const void* tw, cudaStream_t s) {
  constexpr int FS = NX == 2048 ? 2 * 1056 : (NX / 32) * 33;
  constexpr int NTW = NX == 2048 ? 2048 : NX == 1024 ? 1024 : 512;
  const size_t smem = ((size_t)NTW + (size_t)W * FS) * sizeof(float2);
  auto kern = k_xfft_rows<NX, W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid1(nrows, W), 32 * W, smem, s>>>((float2*)data, nrows, (const float2*)tw);
  return cudaGetLastError();
}

cudaError_t launch_xfft_rows(void* data, int nx, long long nrows, const void* tw, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  if (!tw || ((uintptr_t)data & 15)) return cudaErrorInvalidValue;  // 16-byte row copies
  // 8 warps (2 blocks per SM) for 512- and 1024-point rows; 2048-point rows
  // stage 17 KB per warp: 4 warps (2 blocks per SM)
  if (nx == 1024) return xfft_rows_impl<1024, 8>(data, nrows, tw, s);
  if (nx == 2048) return xfft_rows_impl<2048, 4>(data, nrows, tw, s);
  if (nx == 512) return xfft_rows_impl<512, 8>(data, nrows, tw, s);
  return cudaErrorInvalidValue;
}

bool yz_fusable(int nx, int ny, int nz) {
  // 2048 rows: from 4 slices up (a work item re-reads its bin indices from
  // the per-pixel geometry, 4x the bytes of one slice of its tile, which the
  // separate y and z passes beat on thinner stacks: 2048^2 x 1 film 21 ms
  // against 31 ms per energy)
  return (ny == 2048 || ny == 1024 || ny == 512) && nx >= 16 && (nx & (nx - 1)) == 0 &&
         nz >= (ny == 2048 ? 4 : 1) && nz <= 1024 && (nz & (nz - 1)) == 0;
}

// sel.nzfull > 0: the z-first path's planes (nz = their count per field).
static bool yz_sel_ok(int nx, int nz, const YzSel& sel) {
  return nx >= 16 && (nx & (nx - 1)) == 0 && nz >= 1 && nz <= sel.nzfull && sel.nzfull <= 1024 &&
         (sel.nzfull & (sel.nzfull - 1)) == 0 && sel.kb >= 0 && sel.kb < sel.nzfull;
}

cudaError_t launch_yz512_tma(const void* tmap, int nx, int nz, int nf, const Geo<float>* geo,
                             const void* twz, const void* twy, const unsigned short* b0idx,
                             void* part, int* err, int n_sm, unsigned poll, long long* L_out,
                             cudaStream_t s, YzSel sel) {
  const bool is_sel = sel.nzfull > 0;
  if (!(is_sel ? yz_sel_ok(nx, nz, sel) : yz_fusable(nx, 512, nz)) || n_sm <= 0 ||
      (nf != 3 && nf != 5))
    return cudaErrorInvalidValue;
  const long long ntiles = nx / 16, items = nf * ntiles, T = items * nz;
  // equal step ranges over as many blocks as SMs, but at least nz / 3 steps
  // each, so an item meets at most kYzSlots blocks
  const long long L0 = (T + n_sm - 1) / n_sm, Lmin = (nz + kYzSlots - 2) / (kYzSlots - 1);
  const long long L = L0 > Lmin ? L0 : Lmin;
  const long long grid = (T + L - 1) / L;
  // SEL: every bin is stored once, in slot 0 (k_ewald_bins adds no other slot)
  *L_out = is_sel ? T : L;
  const size_t smem = (2 * 8192 + 32 * 33 * 8 + 512 + (size_t)nz) * sizeof(float2) +
                      8192 * sizeof(unsigned short) + 2 * 8;
  auto kern = is_sel ? k_yz512_tma<true> : k_yz512_tma<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)grid, 512, smem, s>>>(*(const CUtensorMap*)tmap, nx, nz, nf, (int)ntiles, (int)L,
                                         (int)T, geo, (const float2*)twz, (const float2*)twy, b0idx,
                                         (float4*)part, err, poll, sel.kb, sel.nzfull - 1);
  return cudaGetLastError();
}

cudaError_t launch_yz_tma(const void* tmap, int nx, int ny, int nz, int nf, const Geo<float>* geo,
                          const void* twz, const void* tw4, const void* tw2k,
                          const unsigned short* b0idx, void* part, int* err, int n_sm,
                          unsigned poll, long long* L_out, cudaStream_t s, YzSel sel) {
  const bool is_sel = sel.nzfull > 0;
  if (!(is_sel ? yz_sel_ok(nx, nz, sel) && (ny == 1024 || ny == 2048) : yz_fusable(nx, ny, nz)) ||
      ny == 512 || n_sm <= 0)
    return cudaErrorInvalidValue;
  if (nf != 3 && nf != 5) return cudaErrorInvalidValue;
  // 1024 rows: pairs of 8-column tiles; 2048 rows: quads of 4-column tiles
  const bool y2k = ny == 2048;
  if (y2k && !tw2k) return cudaErrorInvalidValue;
  const int grp = y2k ? 4 : 2;
  const long long ntiles = y2k ? nx / 4 : nx / 8, items = nf * (ntiles / grp), T = items * nz;
  if (n_sm < grp) return cudaErrorInvalidValue;
  // equal step ranges over as many block groups as SMs allow, but at least
  // nz / 3 steps each, so an item meets at most kYzSlots groups
  const long long P0 = n_sm / grp;
  const long long L0 = (T + P0 - 1) / P0, Lmin = (nz + kYzSlots - 2) / (kYzSlots - 1);
  const long long L = L0 > Lmin ? L0 : Lmin;
  const long long groups = (T + L - 1) / L;
  // SEL: every bin is stored once, in slot 0 (k_ewald_bins adds no other slot)
  *L_out = is_sel ? T : L;
  const size_t smem = (2 * 8192 + 32 * 33 * 8 + 1024 + (size_t)nz) * sizeof(float2) +
                      8192 * sizeof(unsigned short) + 2 * 8;
  auto kern = y2k ? (is_sel ? k_yz_tma<true, true> : k_yz_tma<true, false>)
                  : (is_sel ? k_yz_tma<false, true> : k_yz_tma<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)(grp * groups), 512, smem, s>>>(*(const CUtensorMap*)tmap, nx, nz, nf,
                                                    (int)ntiles, (int)L, (int)T, geo,
                                                    (const float2*)twz, (const float2*)tw4,
                                                    (const float2*)tw2k, b0idx, (float4*)part,
                                                    err, poll, sel.kb, sel.nzfull - 1);
  return cudaGetLastError();
}

cudaError_t launch_bins5_from_part(const void* part, int nx, int ny, int nz, long long L,
                                  const Geo<float>* geo, float dc, void* bins, cudaStream_t s) {
  const long long npix = (long long)nx * ny;
  k_bins5_from_part<<<grid1(npix, 256), 256, 0, s>>>((const float4*)part, nx, ny, nz, nx / 8,
                                                     (int)L, geo, dc, (float2*)bins);
  return cudaGetLastError();
}

cudaError_t launch_ewald_bins(const void* part, int nx, int ny, int nz, long long L,
                              const Geo<float>* geo, float dc0, float dc1, float dc2, float* img,
                              cudaStream_t s) {
  const long long npix = (long long)nx * ny;
  k_ewald_bins<<<grid1(npix, 256), 256, 0, s>>>((const float4*)part, nx, ny, nz, nx / 8, (int)L, geo,
                                                dc0, dc1, dc2, img);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_col_fft4s(void* p, long long S, long long W, const ColBatches& bt,
                             const void* tw4, cudaStream_t s) {
  using C = typename RT<R>::C;
  constexpr int TX = 8;  // 75 KB (FP32) / 151 KB (FP64) of shared memory
  if (W % TX) return cudaErrorInvalidValue;
  const long long ntiles = W / TX;
  const long long total = ntiles * bt.nbatch;
  if (total <= 0) return cudaSuccess;
  const size_t smem = (32 * 33 * TX + 1024) * sizeof(C);
  auto kern = k_col_fft4s<R, TX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)total, 32 * TX, smem, s>>>((C*)p, S, ntiles, bt.bdiv, bt.stride_hi,
                                               bt.stride_lo, bt.base, (const C*)tw4);
  return cudaGetLastError();
}

cudaError_t launch_col_fft4s_tma(const void* tmap, void* p, long long S, long long W,
                                 const ColBatches& bt, const void* tw4, int* err, int n_sm,
                                 unsigned poll, cudaStream_t s) {
  using C = float2;
  constexpr int TX = 8;
  if (W % TX || bt.base != 0) return cudaErrorInvalidValue;
  const long long ntiles = W / TX;
  const long long total = ntiles * bt.nbatch;
  if (total <= 0) return cudaSuccess;
  const size_t smem = (2 * 1024 * TX + 32 * 33 * TX + 1024) * sizeof(C) + 2 * 8;
  auto kern = k_col_fft4s_tma<float>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long grid = total < n_sm ? total : n_sm;
  kern<<<(unsigned)grid, 256, smem, s>>>(*(const CUtensorMap*)tmap, (C*)p, S, ntiles, total,
                                         bt.bdiv, bt.stride_hi, bt.stride_lo, (const C*)tw4, err, poll);
  return cudaGetLastError();
}

template <typename R, int T, int EC>
static cudaError_t row_fft_impl(void* p, int nx, long long nrows, const void* twx, cudaStream_t s,
                                const void* src) {
  using C = typename RT<R>::C;
  size_t smem = padded(EC) * sizeof(C);
  int tw_in_smem = 0;
  if (smem + nx * sizeof(C) <= 200 * 1024) {
    smem += nx * sizeof(C);
    tw_in_smem = 1;
  }
  auto kern = k_row_fft<R, T, EC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid1(nrows, EC / nx), T, smem, s>>>((const C*)(src ? src : p), (C*)p, ilog2(nx), nrows,
                                               (const C*)twx, tw_in_smem);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_row_fft4s(void* p, long long nrows, const void* tw4, cudaStream_t s,
                             const void* src) {
  using C = typename RT<R>::C;
  constexpr int W = 8;
  if (nrows <= 0) return cudaSuccess;
  const size_t smem = (1024 + W * 32 * 33) * sizeof(C);
  auto kern = k_row_fft4s<R, W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid1(nrows, W), 32 * W, smem, s>>>((const C*)(src ? src : p), (C*)p, nrows,
                                              (const C*)tw4);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_row_fft(void* p, int nx, long long nrows, const void* twx, cudaStream_t s,
                           const void* src) {
  if (nx & (nx - 1)) {  // any other length: the mixed-radix passes
    const AnyLines ln = {nrows, 1, 1, nx, 0, 0, 0, 1};
    return launch_fft_any<R>(src ? src : p, p, nx, ln, twx, s);
  }
  if (nx <= 2048) return row_fft_impl<R, 256, 2048>(p, nx, nrows, twx, s, src);
  return row_fft_impl<R, 256, 4096>(p, nx, nrows, twx, s, src);
}

template <typename R, int T, int EC, int LOGL, int MINB = 3>
static cudaError_t col_fft_impl(void* p, int L, long long S, long long W, const ColBatches& bt,
                                const void* tw, cudaStream_t s) {
  using C = typename RT<R>::C;
  if (L > EC) return cudaErrorInvalidValue;
  long long TX = EC / L;
  if (TX > W) TX = W;
  if (TX < 1) TX = 1;
  if (LOGL >= 0 && TX != EC / L) return cudaErrorInvalidValue;
  const int logTX = ilog2(TX);
  const long long ntiles = W / TX;
  const long long total = ntiles * bt.nbatch;
  if (total <= 0) return cudaSuccess;
  size_t smem = (size_t)padded(EC) * sizeof(C);
  int tw_in_smem = 0;
  if (smem + L * sizeof(C) <= 200 * 1024) {
    smem += L * sizeof(C);
    tw_in_smem = 1;
  }
  auto kern = k_col_fft<R, T, EC, LOGL, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)total, T, smem, s>>>((C*)p, ilog2(L), S, logTX, ntiles, bt.bdiv, bt.stride_hi,
                                        bt.stride_lo, bt.base, (const C*)tw, tw_in_smem);
  return cudaGetLastError();
}

template <typename R, int EC>
static cudaError_t col_fft_dispatch(void* p, int L, long long S, long long W, const ColBatches& bt,
                                    const void* tw, cudaStream_t s) {
  const int logL = ilog2(L);
  if (W >= EC / L) {
    switch (logL) {
#define RSX_COL(LL) \
  case LL: return col_fft_impl<R, 256, EC, LL>(p, L, S, W, bt, tw, s);
      RSX_COL(5) RSX_COL(6) RSX_COL(7) RSX_COL(8) RSX_COL(9) RSX_COL(10) RSX_COL(11) RSX_COL(12)
#undef RSX_COL
      default: break;
    }
  }
  return col_fft_impl<R, 256, EC, -1>(p, L, S, W, bt, tw, s);
}

template <typename R>
cudaError_t launch_col_fft(void* p, int L, long long S, long long W, const ColBatches& bt,
                           const void* tw, cudaStream_t s) {
  if (L == 1) return cudaSuccess;
  // the Stockham column kernels take power-of-two lengths and row widths
  // (their tiles are power-of-two column groups); anything else takes the
  // mixed-radix passes
  if ((L & (L - 1)) || (W & (W - 1))) {
    const AnyLines ln = {bt.nbatch * W, W, bt.bdiv, bt.stride_hi, bt.stride_lo, bt.base, 1, S};
    return launch_fft_any<R>(p, p, L, ln, tw, s);
  }
  // FP32 2048-point columns: the four-step kernel on 8-column tiles (64-byte
  // row segments, ~146 KB of shared memory, one 512-thread CTA per SM; the
  // 4-column variant, two CTAs per SM, measured 10 % slower), tw the
  // 2048-entry table
  if (sizeof(R) == 4 && L == 2048 && W % 8 == 0) {
    constexpr int TX = 8;
    const long long ntiles = W / TX, total = ntiles * bt.nbatch;
    if (total <= 0) return cudaSuccess;
    const size_t smem = (32 * (64 * TX + TX) + 2048) * sizeof(float2);
    auto kern = k_col_fft2k<TX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)total, 64 * TX, smem, s>>>((float2*)p, S, ntiles, bt.bdiv, bt.stride_hi,
                                                bt.stride_lo, bt.base, (const float2*)tw);
    return cudaGetLastError();
  }
  // 4096 elements per CTA: 34 KB (FP32) or 70 KB (FP64) of padded tile
  return col_fft_dispatch<R, 4096>(p, L, S, W, bt, tw, s);
}

// Radices for length n: 16s, then the rest of the power of two, then 7, 5,
// 3, then the remaining primes (each its own O(p^2) pass).
static AnyPlan any_plan(int n) {
  AnyPlan pl;
  memset(&pl, 0, sizeof(pl));
  pl.n = n;
  int m = n;
  const int small[] = {16, 8, 4, 2, 7, 5, 3};
  for (int r : small)
    while (m % r == 0 && pl.np < kAnyMaxPass) pl.rad[pl.np++] = r, m /= r;
  for (int p = 11; p * p <= m && pl.np < kAnyMaxPass; p += 2)
    while (m % p == 0 && pl.np < kAnyMaxPass) pl.rad[pl.np++] = p, m /= p;
  if (m > 1 && pl.np < kAnyMaxPass) pl.rad[pl.np++] = m, m = 1;
  if (m != 1) pl.np = -1;  // not reachable for n <= 4096
  return pl;
}

template <typename R>
cudaError_t launch_fft_any(const void* src, void* dst, int n, const AnyLines& ln, const void* tw,
                           cudaStream_t s) {
  using C = typename RT<R>::C;
  if (n < 1 || n > 4096 || ln.W < 1 || ln.bdiv < 1) return cudaErrorInvalidValue;
  if (ln.nlines <= 0) return cudaSuccess;
  const AnyPlan pl = any_plan(n);
  if (pl.np < 0) return cudaErrorInvalidValue;
  // both buffers hold at most 2 x 4096 elements; up to 64 lines per CTA
  long long lpc = 4096 / n;
  if (lpc < 1) lpc = 1;
  if (lpc > 64) lpc = 64;
  if (lpc > ln.nlines) lpc = ln.nlines;
  const size_t smem = (2 * (size_t)lpc * n + n) * sizeof(C);
  auto kern = k_fft_any<R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int lines_fast = ln.estride != 1 && ln.xstride == 1;
  kern<<<grid1(ln.nlines, (int)lpc), 256, smem, s>>>((const C*)src, (C*)dst, pl, ln, (int)lpc,
                                                     lines_fast, (const C*)tw);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_dft_z(const void* in, void* out, int nx, int ny, int nz, const void* twz,
                         cudaStream_t s) {
  using C = typename RT<R>::C;
  const long long npix = (long long)nx * ny;
  const long long total = 3 * npix * nz;
  k_dft_z<R><<<grid1(total, 256), 256, 0, s>>>((const C*)in, (C*)out, npix, nz, (const C*)twz);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_geometry(Geo<R>* geo, int nx, int ny, int nz, double voxel_nm, double k,
                            cudaStream_t s, unsigned short* b0idx) {
  k_geometry<R><<<grid1((long long)nx * ny, 256), 256, 0, s>>>(geo, nx, ny, nz, voxel_nm, k,
                                                               b0idx);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ewald(const void* p, int nx, int ny, int nz, const Geo<R>* geo,
                         const void* twz, bool pruned, const R dc[3], void* img, cudaStream_t s,
                         int* err, unsigned poll) {
  using C = typename RT<R>::C;
  const long long npix = (long long)nx * ny;
  if (!pruned) {
    k_ewald_full<R><<<grid1(npix, 256), 256, 0, s>>>((const C*)p, nx, ny, nz, geo, (R*)img);
    return cudaGetLastError();
  }
  if (npix % 2) {
    k_ewald_each<R><<<grid1(npix, 256), 256, 0, s>>>((const C*)p, nx, ny, nz, geo, (const C*)twz,
                                                     dc[0], dc[1], dc[2], (R*)img);
    return cudaGetLastError();
  }
  constexpr int PX = 512, S = 4;
  if (err && npix % PX == 0 && nz <= 4096) {
    const size_t smem = (size_t)S * 3 * PX * sizeof(C) + S * 8 + (size_t)nz * sizeof(C);
    auto kern = k_ewald_tma<R, PX, S>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)(npix / PX), PX / 2, smem, s>>>((const C*)p, nx, ny, nz, geo, (const C*)twz,
                                                     dc[0], dc[1], dc[2], (R*)img, err, poll);
    return cudaGetLastError();
  }
  const int tw_in_smem = nz <= 4096;
  const size_t smem = tw_in_smem ? nz * sizeof(C) : 0;
  auto kern = k_ewald_pruned<R, 4>;
  // FP64 tables above 3072 entries exceed the 48 KB default
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid1(npix / 2, 256), 256, smem, s>>>((const C*)p, nx, ny, nz, geo, (const C*)twz,
                                               tw_in_smem, dc[0], dc[1], dc[2], (R*)img);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_zbins5(const void* f, int nx, int ny, int nz, const Geo<R>* geo, const void* twz,
                          double dc, void* bins, cudaStream_t s) {
  using C = typename RT<R>::C;
  const long long npix = (long long)nx * ny;
  const int tw_in_smem = nz <= 4096;
  const size_t smem = tw_in_smem ? nz * sizeof(C) : 0;
  auto kern = k_zbins5<R, 4>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid1(npix, 256), 256, smem, s>>>((const C*)f, nx, ny, nz, geo, (const C*)twz, tw_in_smem,
                                           (R)dc, (C*)bins);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ewald_linear(const void* bins, int nx, int ny, const Geo<R>* geo, double alpha,
                                bool literal, void* img, cudaStream_t s) {
  using C = typename RT<R>::C;
  k_ewald_linear<R><<<grid1((long long)nx * ny, 256), 256, 0, s>>>(
      (const C*)bins, nx, ny, geo, (R)cos(alpha), (R)sin(alpha), literal ? 1 : 0, (R*)img);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_nt_all(const void* M, long long N, const PolParams<R>& pp, void* nt,
                          cudaStream_t s) {
  k_nt_all<R><<<grid1(N, 256), 256, 0, s>>>((const typename RT<R>::V4*)M, N, pp,
                                            (typename RT<R>::C*)nt);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_nt_comp(const void* Mj, long long off, long long n, long long N, int j,
                           bool first, const PolParams<R>& pp, void* nt, cudaStream_t s) {
  using V4 = typename RT<R>::V4;
  using C = typename RT<R>::C;
  if (n <= 0) return cudaSuccess;
  if (first)
    k_nt_comp<R, true><<<grid1(n, 256), 256, 0, s>>>((const V4*)Mj, off, n, N, j, pp, (C*)nt);
  else
    k_nt_comp<R, false><<<grid1(n, 256), 256, 0, s>>>((const V4*)Mj, off, n, N, j, pp, (C*)nt);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_nt_restore(const void* nt, void* out, long long N, double ref, cudaStream_t s) {
  using C = typename RT<R>::C;
  k_nt_restore<R><<<grid1(5 * N, 256), 256, 0, s>>>((const C*)nt, (C*)out, N, (R)ref);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_rotate_acc(const void* img, void* acc, int nx, int ny, double alpha,
                              bool rotate, cudaStream_t s) {
  long long c[4];
  rotation_coeffs(alpha, nx, ny, c);
  const dim3 block(kRotTile, kRotTile);
  const dim3 grid((nx + kRotTile - 1) / kRotTile, (ny + kRotTile - 1) / kRotTile);
  k_rotate_acc<R><<<grid, block, 0, s>>>((const R*)img, (R*)acc, nx, ny, c[0], c[1], c[2], c[3],
                                          rotate ? 1 : 0);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ewald_linear_many(const void* bins, int nx, int ny, const Geo<R>* geo,
                                     const AngleBatch<R>& ab, bool literal, void* imgs,
                                     cudaStream_t s) {
  if (ab.n <= 0) return cudaSuccess;
  if (ab.n > kMaxAngleBatch) return cudaErrorInvalidValue;
  const long long npix = (long long)nx * ny;
  const dim3 grid(grid1(npix, 256), ab.n);
  k_ewald_linear_many<R><<<grid, 256, 0, s>>>((const typename RT<R>::C*)bins, nx, ny, geo, ab,
                                              literal ? 1 : 0, (R*)imgs);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_rotate_acc_many(const void* imgs, void* acc, int nx, int ny,
                                   const AngleBatch<R>& ab, bool rotate, cudaStream_t s) {
  if (ab.n <= 0) return cudaSuccess;
  if (ab.n > kMaxAngleBatch) return cudaErrorInvalidValue;
  const dim3 block(kRotTile, kRotTile);
  const dim3 grid((nx + kRotTile - 1) / kRotTile, (ny + kRotTile - 1) / kRotTile);
  k_rotate_acc_many<R><<<grid, block, 0, s>>>((const R*)imgs, (R*)acc, nx, ny, ab,
                                               rotate ? 1 : 0);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_scale(const void* acc, void* out, long long n, double scale, cudaStream_t s) {
  k_scale<R><<<grid1(n, 256), 256, 0, s>>>((const R*)acc, (R*)out, n, (R)scale);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_validate(const void* M, long long n_entries, int* flag, cudaStream_t s) {
  if (n_entries == 0) return cudaSuccess;
  k_validate<R><<<grid1(n_entries, 256), 256, 0, s>>>((const R*)M, n_entries, flag);
  return cudaGetLastError();
}

#define RSX_INSTANTIATE(R)                                                                        \
  template cudaError_t launch_pol_fftx<R>(const void*, int, int, int, const PolParams<R>&, bool,  \
                                          void*, const void*, cudaStream_t, long long, long long, \
                                          const void*);                                          \
  template cudaError_t launch_director<R>(const void*, long long, long long, void*, cudaStream_t);\
  template cudaError_t launch_row_fft<R>(void*, int, long long, const void*, cudaStream_t,         \
                                         const void*);                                           \
  template cudaError_t launch_row_fft4s<R>(void*, long long, const void*, cudaStream_t,           \
                                           const void*);                                         \
  template cudaError_t launch_col_fft<R>(void*, int, long long, long long, const ColBatches&,     \
                                         const void*, cudaStream_t);                              \
  template cudaError_t launch_dft_z<R>(const void*, void*, int, int, int, const void*,            \
                                       cudaStream_t);                                             \
  template cudaError_t launch_fft_any<R>(const void*, void*, int, const AnyLines&, const void*,   \
                                         cudaStream_t);                                           \
  template cudaError_t launch_geometry<R>(Geo<R>*, int, int, int, double, double, cudaStream_t,  \
                                          unsigned short*);                                      \
  template cudaError_t launch_ewald<R>(const void*, int, int, int, const Geo<R>*, const void*,     \
                                       bool, const R*, void*, cudaStream_t, int*, unsigned);      \
  template cudaError_t launch_rotate_acc<R>(const void*, void*, int, int, double, bool,           \
                                            cudaStream_t);                                        \
  template cudaError_t launch_ewald_linear_many<R>(const void*, int, int, const Geo<R>*,          \
                                                   const AngleBatch<R>&, bool, void*,            \
                                                   cudaStream_t);                                 \
  template cudaError_t launch_rotate_acc_many<R>(const void*, void*, int, int,                    \
                                                 const AngleBatch<R>&, bool, cudaStream_t);      \
  template cudaError_t launch_scale<R>(const void*, void*, long long, double, cudaStream_t);      \
  template cudaError_t launch_validate<R>(const void*, long long, int*, cudaStream_t);          \
  template cudaError_t launch_ntp_fftx<R>(const void*, int, int, int, const PolParams<R>&, bool,  \
                                          void*, const void*, cudaStream_t, long long, long long);\
  template cudaError_t launch_nt_all<R>(const void*, long long, const PolParams<R>&, void*,       \
                                        cudaStream_t);                                            \
  template cudaError_t launch_nt_comp<R>(const void*, long long, long long, long long, int, bool, \
                                         const PolParams<R>&, void*, cudaStream_t);               \
  template cudaError_t launch_nt_restore<R>(const void*, void*, long long, double, cudaStream_t); \
  template cudaError_t launch_pol_fft4s<R>(const void*, const void*, int, int, int,               \
                                           const PolParams<R>&, void*, const void*, cudaStream_t, \
                                           const void*);                                         \
  template cudaError_t launch_col_fft4s<R>(void*, long long, long long, const ColBatches&,         \
                                           const void*, cudaStream_t);                            \
  template cudaError_t launch_zbins5<R>(const void*, int, int, int, const Geo<R>*, const void*,    \
                                        double, void*, cudaStream_t);                             \
  template cudaError_t launch_ewald_linear<R>(const void*, int, int, const Geo<R>*, double, bool,  \
                                              void*, cudaStream_t);


RSX_INSTANTIATE(float)
RSX_INSTANTIATE(double)

}  // namespace rsx
