// Internal (C++) interface between the C ABI layer and the CUDA kernels.
#pragma once

#include <math.h>

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/rsx.h"

namespace rsx {

// Per-energy, per-angle constants of Eq. (polarization), in the split form
// that keeps FP32 accurate: with eps = n - 1 (small, Sec. 3.2),
//   tau   = (eps_par + 2 eps_perp) / 3          (Tr(N)/3 - 1)
//   dperp = eps_perp - tau                      (n_perp - Tr(N)/3)
//   dpar  = eps_par - eps_perp                  (n_par - n_perp)
// Complex values are stored as (re, im) pairs of R.
template <typename R> struct PolParams {
  R tau[RSX_MAX_COMPONENTS][2];
  R dperp[RSX_MAX_COMPONENTS][2];
  R dpar[RSX_MAX_COMPONENTS][2];
  // Per component, complex, from the three above: tau (2 + tau),
  // 2 dperp (1 + tau), dperp^2, 2 dpar (1 + tau), dpar (2 dperp + dpar).
  // With tau' = tau + s dperp: tau' (2 + tau') = q0 + s q1 + s^2 q2 and
  // (v s dpar) (2 v (1 + tau') + v s dpar) = v^2 (s q3 + s^2 q4).
  R q[RSX_MAX_COMPONENTS][5][2];
  R ce, se;     // cos(alpha), sin(alpha): e = U(alpha) (1, 0, 0)
  int c;        // number of components
  int literal;  // 1: p <- U^T p (RSX_FRAME_LITERAL), 0: lab frame
  int add_ref;  // 1: output full p; 0: p minus the constant -(c-1) e'/(4 pi)
};

// Polls of an mbarrier before a pipelined kernel gives up on a copy (the
// default; a context may lower it to exercise the failure path).  Waits that
// drain copies in flight before a block exits always use this bound.
constexpr unsigned kWaitPolls = 1u << 22;

// A batch of e-field angles for the linearity path's per-angle passes:
// cos, sin of alpha and the detector rotation's fixed-point coefficients
// (2^-48) of Q -> U(alpha) Q in pixel units.
constexpr int kMaxAngleBatch = 64;
template <typename R> struct AngleBatch {
  int n;
  R ce[kMaxAngleBatch], se[kMaxAngleBatch];
  long long cxx[kMaxAngleBatch], cxy[kMaxAngleBatch], cyx[kMaxAngleBatch], cyy[kMaxAngleBatch];
};

// fx = cx + cos a dx - sin a (nx/ny) dy, fy = cy + sin a (ny/nx) dx + cos a dy
inline void rotation_coeffs(double alpha, int nx, int ny, long long c[4]) {
  const double two48 = 281474976710656.0;
  const double ca = cos(alpha), sa = sin(alpha);
  c[0] = llround(ca * two48);
  c[1] = llround(sa * ((double)nx / ny) * two48);
  c[2] = llround(sa * ((double)ny / nx) * two48);
  c[3] = c[0];
}

template <typename R>
inline void add_angle(AngleBatch<R>& ab, double alpha, int nx, int ny) {
  long long c[4];
  rotation_coeffs(alpha, nx, ny, c);
  const int a = ab.n++;
  ab.ce[a] = (R)cos(alpha);
  ab.se[a] = (R)sin(alpha);
  ab.cxx[a] = c[0];
  ab.cxy[a] = c[1];
  ab.cyx[a] = c[2];
  ab.cyy[a] = c[3];
}

// Component j of pp from tau = (eps_par + 2 eps_perp)/3, dperp = eps_perp -
// tau and dpar = eps_par - eps_perp (complex, eps = n - 1), in FP64.
template <typename R>
inline void set_component(PolParams<R>& pp, int j, double tr, double ti, double pr, double pi,
                          double ar, double ai) {
  pp.tau[j][0] = (R)tr;
  pp.tau[j][1] = (R)ti;
  pp.dperp[j][0] = (R)pr;
  pp.dperp[j][1] = (R)pi;
  pp.dpar[j][0] = (R)ar;
  pp.dpar[j][1] = (R)ai;
  const double q[5][2] = {
      {tr * (2.0 + tr) - ti * ti, ti * (2.0 + tr) + tr * ti},
      {2.0 * (pr * (1.0 + tr) - pi * ti), 2.0 * (pi * (1.0 + tr) + pr * ti)},
      {pr * pr - pi * pi, 2.0 * pr * pi},
      {2.0 * (ar * (1.0 + tr) - ai * ti), 2.0 * (ai * (1.0 + tr) + ar * ti)},
      {ar * (2.0 * pr + ar) - ai * (2.0 * pi + ai), ai * (2.0 * pr + ar) + ar * (2.0 * pi + ai)}};
  for (int k = 0; k < 5; ++k) {
    pp.q[j][k][0] = (R)q[k][0];
    pp.q[j][k][1] = (R)q[k][1];
  }
}

// Per-pixel Ewald geometry for one energy (Eq. Ewald): the two bracketing
// q_z bins (b0 < 0 marks a pixel with no real q_z), the interpolation
// weight w of bin b1, r-hat = k_out/|k_out| and |k_out|^4.
template <typename R> struct __align__(16) Geo {
  int b0, b1;
  R w, rx, ry, rz, k4;
};

// Batches of a column-FFT launch: batch b starts at
// base + (b / bdiv) * stride_hi + (b % bdiv) * stride_lo (complex elements).
struct ColBatches {
  long long nbatch, bdiv, stride_hi, stride_lo, base;
};

// Sets the message returned by rsx_last_error() on this host thread.
void set_last_error(const char* msg);

// RSX_OK when p is device memory of device `dev` or managed memory;
// otherwise sets the message (naming `what`) and returns RSX_ERR_INVALID.
// Uses cudaPointerGetAttributes, which allocates nothing.
int check_device_pointer(const void* p, int dev, const char* what);

// Rows are (z, y) pairs; row_begin / row_count restrict the launch to a
// range of rows (a group of z-slices); row_count < 0 means all rows.
// dir: the morphology's cached director ([c][3][N] Real, launch_director)
// or nullptr (computed from phi and theta).
template <typename R>
cudaError_t launch_pol_fftx(const void* M, int nx, int ny, int nz, const PolParams<R>& pp,
                            bool do_fft, void* p, const void* twx, cudaStream_t s,
                            long long row_begin = 0, long long row_count = -1,
                            const void* dir = nullptr);
// The director of every component and voxel, dir[c][3][N], from M
// (n_entries = c N).
template <typename R>
cudaError_t launch_director(const void* M, long long n_entries, long long N, void* dir,
                            cudaStream_t s);
// Algorithm 2: p = N_t . e from nt[5][N] (xx, xy, yy, xz, yz), fused with
// the x-FFT like launch_pol_fftx.
template <typename R>
cudaError_t launch_ntp_fftx(const void* nt, int nx, int ny, int nz, const PolParams<R>& pp,
                            bool do_fft, void* p, const void* twx, cudaStream_t s,
                            long long row_begin = 0, long long row_count = -1);
// Algorithm 3: N_t from device-resident M (all components), or one
// component's staged voxel range [off, off + n) added to it.
template <typename R>
cudaError_t launch_nt_all(const void* M, long long N, const PolParams<R>& pp, void* nt,
                          cudaStream_t s);
template <typename R>
cudaError_t launch_nt_comp(const void* Mj, long long off, long long n, long long N, int j,
                           bool first, const PolParams<R>& pp, void* nt, cudaStream_t s);
template <typename R>
cudaError_t launch_nt_restore(const void* nt, void* out, long long N, double ref, cudaStream_t s);
// Linearity fast path: the two q_z bins of the five FFT'd N_t entries per
// pixel (f[5][N] -> bins[5][2][npix]), then one angle's image from them.
template <typename R>
cudaError_t launch_zbins5(const void* f, int nx, int ny, int nz, const Geo<R>* geo, const void* twz,
                          double dc, void* bins, cudaStream_t s);
template <typename R>
cudaError_t launch_ewald_linear(const void* bins, int nx, int ny, const Geo<R>* geo, double alpha,
                                bool literal, void* img, cudaStream_t s);
// Four-step (32 x 32) transforms for 1024-point axes: the x pass fused with
// the polarisation (from M, or from N_t when nt is given) and the y pass.
// tw4[k2 * 32 + n1] = exp(-2 pi i n1 k2 / 1024).
template <typename R>
cudaError_t launch_pol_fft4s(const void* M, const void* nt, int nx, int ny, int nz,
                             const PolParams<R>& pp, void* p, const void* tw4, cudaStream_t s,
                             const void* dir = nullptr);
template <typename R>
cudaError_t launch_col_fft4s(void* p, long long S, long long W, const ColBatches& bt,
                             const void* tw4, cudaStream_t s);
// The Algorithm-1 x pass (FP32, nx = 1024 or 512) streaming the morphology
// through a ring of bulk-copy stages into warp-specialised blocks
// (polarisation, transform, producer); M must be 16-byte aligned; two
// persistent CTAs per SM (n_sm).  tw: the four-step table W1024^(ab) as
// [32][32] for nx = 1024, the 512-point table W512^j for nx = 512.
cudaError_t launch_pol_fft4s_tma(const void* M, int nx, int ny, int nz, const PolParams<float>& pp,
                                 void* p, const void* tw4, int* err, int n_sm, unsigned poll,
                                 cudaStream_t s);
// Up to kMaxXAngles e-field angles for one multi-angle x pass (which takes
// up to 8) or z-first pass: cos and sin of each, n of them in use.
constexpr int kMaxXAngles = 32;
struct XAngles {
  float ce[kMaxXAngles], se[kMaxXAngles];
  int n;
};
// The Algorithm-1 x pass for ang.n angles per read of the morphology (FP32,
// nx = 1024 or 512, M 16-byte aligned): angle k's three x-transformed fields
// go to p + k * pstride (complex elements; pstride >= 3 N).  pp supplies the
// optical constants and the frame (its ce, se are not used).  One persistent
// CTA per SM (n_sm).
cudaError_t launch_pol_fft4s_tma_multi(const void* M, int nx, int ny, int nz,
                                       const PolParams<float>& pp, const XAngles& ang, void* p,
                                       long long pstride, const void* tw, int* err, int n_sm,
                                       unsigned poll, cudaStream_t s);
// The z-first Algorithm 1 pass (FP32): p for ang.n angles per read of the
// morphology, each pixel's z column transformed, and only the ns bins
// kb .. kb + ns - 1 (mod nz) kept: angle k's plane s of field f goes to
// out + k * kstride + f * fstride + s * nx * ny as an [ny][nx] complex plane
// (not yet x- or y-transformed).  tmap: a CUtensorMap over the morphology
// viewed as [c nz][ny][4 nx] floats with (128 / nz) x 1 x nz boxes (see
// make_tmap_m); twz: exp(-2 pi i j / nz), j < nz.  zfirst_fusable says
// whether the shape qualifies (nz = 32, 64 or 128; nx and ny = 512, 1024 or
// 2048).  One persistent CTA per SM (n_sm).
bool zfirst_fusable(int nx, int ny, int nz);
cudaError_t launch_pol_zfft_multi(const void* tmap, int nx, int ny, int nz,
                                  const PolParams<float>& pp, const XAngles& ang, void* out,
                                  long long kstride, long long fstride, int kb, int ns,
                                  const void* twz, int* err, int n_sm, unsigned poll,
                                  cudaStream_t s);
// In-place x-FFT of nrows contiguous rows of nx = 512, 1024 or 2048 complex
// (FP32; tw: twx for 512, tw4 for 1024, the 2048-point table for 2048).
cudaError_t launch_xfft_rows(void* data, int nx, long long nrows, const void* tw, cudaStream_t s);
// The same pipeline for Algorithm 2: p = N_t e from the five stored entries
// of N_t ([5][N] complex float, 16-byte aligned; the reference constant
// left out as k_nt_all stores it).
cudaError_t launch_ntp_fft4s_tma(const void* nt, int nx, int ny, int nz,
                                 const PolParams<float>& pp, void* p, const void* tw4, int* err,
                                 int n_sm, unsigned poll, cudaStream_t s);
// The y-FFT fused with the pruned z transform (FP32): yz_fusable says
// whether the shape qualifies (ny = 2048, 1024 or 512, nx a power of two of
// at least 16, nz a power of two up to 1024, and at least 4 for 2048 rows).
// launch_yz_tma (ny = 1024 or 2048) writes the two q_z bins of every pixel
// and of each of the nf fields (3: p; 5: the linearity path's N_t entries)
// into part ([kYzSlots][nf][ny][nx] float4 = bin b0, bin b0 + 1) and returns
// in *L_out the step count per block that launch_ewald_bins needs to add the
// slots.  tw2k: exp(-2 pi i j / 2048) (ny = 2048 only).
bool yz_fusable(int nx, int ny, int nz);
// Partial-bin slots of the fused pass: a work item's z-slices meet at most
// this many blocks (their step ranges hold at least nz / (kYzSlots - 1)).
constexpr int kYzSlots = 4;
// b0idx: each pixel's lower q_z bin (launch_geometry's packed output).
// sel: the z-first path's planes instead of z-slices when nzfull > 0: nz is
// then the plane count per field (any value up to nzfull), plane s holds bin
// (kb + s) mod nzfull, and each pixel takes its two bins from planes
// (b0 - kb) mod nzfull and the one after.
struct YzSel {
  int kb = 0, nzfull = 0;
};
cudaError_t launch_yz_tma(const void* tmap, int nx, int ny, int nz, int nf, const Geo<float>* geo,
                          const void* twz, const void* tw4, const void* tw2k,
                          const unsigned short* b0idx, void* part, int* err, int n_sm,
                          unsigned poll, long long* L_out, cudaStream_t s, YzSel sel = YzSel());
// The same for ny = 512 (16-column tiles, tensor map boxes of 32 floats x
// 256 rows; twy the 512-point twiddle table).
cudaError_t launch_yz512_tma(const void* tmap, int nx, int nz, int nf, const Geo<float>* geo,
                             const void* twz, const void* twy, const unsigned short* b0idx,
                             void* part, int* err, int n_sm, unsigned poll, long long* L_out,
                             cudaStream_t s, YzSel sel = YzSel());
// The linearity path's per-energy bins (k_zbins5 layout) from launch_yz_tma
// run over the five FFT'd N_t entries (nf = 5); dc = -(c-1)/(4 pi) N.
cudaError_t launch_bins5_from_part(const void* part, int nx, int ny, int nz, long long L,
                                  const Geo<float>* geo, float dc, void* bins, cudaStream_t s);
cudaError_t launch_ewald_bins(const void* part, int nx, int ny, int nz, long long L,
                              const Geo<float>* geo, float dc0, float dc1, float dc2, float* img,
                              cudaStream_t s);
// The y pass with 2-D tensor (TMA) loads, FP32, ny = 1024, whole-volume
// batches (bt.base = 0): tmap is a CUtensorMap over the data viewed as
// [nbatch][ny][2 nx] floats with 16 x 256 x 1 boxes; one persistent CTA per
// SM (n_sm).
cudaError_t launch_col_fft4s_tma(const void* tmap, void* p, long long S, long long W,
                                 const ColBatches& bt, const void* tw4, int* err, int n_sm,
                                 unsigned poll, cudaStream_t s);
// Lines of a general-size FFT launch: line l = (b, x) with b = l / W and
// x = l mod W starts at base + (b / bdiv) stride_hi + (b mod bdiv) stride_lo +
// x xstride and holds its n elements estride apart (complex elements).
struct AnyLines {
  long long nlines, W, bdiv, stride_hi, stride_lo, base, xstride, estride;
};
// Forward, unnormalised DFTs of any length n in [1, 4096] along every line
// (mixed-radix Stockham passes in shared memory), from src to dst (the same
// buffer, or disjoint ones); tw[t] = exp(-2 pi i t / n).
template <typename R>
cudaError_t launch_fft_any(const void* src, void* dst, int n, const AnyLines& lines,
                           const void* tw, cudaStream_t s);
template <typename R>
cudaError_t launch_row_fft(void* p, int nx, long long nrows, const void* twx, cudaStream_t s,
                           const void* src = nullptr);
// 1024-point row FFTs (four-step, one warp per row) from src (or p) to p;
// tw4 the four-step twiddle table.
template <typename R>
cudaError_t launch_row_fft4s(void* p, long long nrows, const void* tw4, cudaStream_t s,
                             const void* src = nullptr);
template <typename R>
cudaError_t launch_col_fft(void* p, int L, long long S, long long W, const ColBatches& bt,
                           const void* tw, cudaStream_t s);
template <typename R>
cudaError_t launch_dft_z(const void* in, void* out, int nx, int ny, int nz, const void* twz,
                         cudaStream_t s);
// b0idx (optional): also each pixel's lower q_z bin as unsigned short (0
// off the sphere), for the fused y+z passes.
template <typename R>
cudaError_t launch_geometry(Geo<R>* geo, int nx, int ny, int nz, double voxel_nm, double k,
                            cudaStream_t s, unsigned short* b0idx = nullptr);
// err: device int that records a pipeline timeout (the bulk-copy pipeline
// of the pruned path is used only when err is given and npix is a multiple
// of 512).
template <typename R>
cudaError_t launch_ewald(const void* p, int nx, int ny, int nz, const Geo<R>* geo,
                         const void* twz, bool pruned, const R dc[3], void* img, cudaStream_t s,
                         int* err = nullptr, unsigned poll = kWaitPolls);
// The linearity path's per-angle passes for a batch of angles: images of
// every angle into imgs ([ab.n][ny][nx], fftshift order), then one
// rotate-and-accumulate pass over all of them (same sums, same order as one
// launch per angle).
template <typename R>
cudaError_t launch_ewald_linear_many(const void* bins, int nx, int ny, const Geo<R>* geo,
                                     const AngleBatch<R>& ab, bool literal, void* imgs,
                                     cudaStream_t s);
template <typename R>
cudaError_t launch_rotate_acc_many(const void* imgs, void* acc, int nx, int ny,
                                   const AngleBatch<R>& ab, bool rotate, cudaStream_t s);
template <typename R>
cudaError_t launch_rotate_acc(const void* img, void* acc, int nx, int ny, double alpha,
                              bool rotate, cudaStream_t s);
template <typename R>
cudaError_t launch_scale(const void* acc, void* out, long long n, double scale, cudaStream_t s);
template <typename R>
cudaError_t launch_validate(const void* M, long long n_entries, int* flag, cudaStream_t s);

}  // namespace rsx
