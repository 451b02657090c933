// C ABI of the GB300 P-RSoXS path (include/rsx.h): context lifetime,
// argument checks and the host-side loops of Algorithm 1 (energies outer,
// e-field angles inner), enqueuing the kernels of rsx_kernels.cu.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/rsx.h"
#include "rsx_kernels.h"

using rsx::Geo;
using rsx::PolParams;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(RSX_ERR_OOM, "%s: out of device memory", what);
  return fail(RSX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define RSX_CK(call, what)                      \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

const double kPi = 3.14159265358979323846264338327950288;
const double kHcEvNm = 1239.84198;  // lambda = hc / E

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int check_config(const rsx_config* c) {
  if (!c) return fail(RSX_ERR_INVALID, "config is NULL");
  if (c->nx < 1 || c->nx > 4096 || c->ny < 1 || c->ny > 4096)
    return fail(RSX_ERR_INVALID, "nx=%d, ny=%d: each must lie in [1, 4096]", c->nx, c->ny);
  if (c->nz < 1 || c->nz > 65535) return fail(RSX_ERR_INVALID, "nz=%d outside [1, 65535]", c->nz);
  if (c->n_components < 1 || c->n_components > RSX_MAX_COMPONENTS)
    return fail(RSX_ERR_INVALID, "n_components=%d outside [1, %d]", c->n_components,
                RSX_MAX_COMPONENTS);
  if (!(c->voxel_nm > 0.0) || !isfinite(c->voxel_nm))
    return fail(RSX_ERR_INVALID, "voxel_nm must be positive and finite");
  if (c->precision != 32 && c->precision != 64)
    return fail(RSX_ERR_INVALID, "precision=%d: must be 32 or 64", c->precision);
  if (c->algorithm < 1 || c->algorithm > 3)
    return fail(RSX_ERR_INVALID, "algorithm=%d: must be 1, 2 or 3", c->algorithm);
  if (c->frame != RSX_FRAME_LITERAL && c->frame != RSX_FRAME_LAB)
    return fail(RSX_ERR_INVALID, "frame=%d: must be RSX_FRAME_LITERAL or RSX_FRAME_LAB", c->frame);
  if (c->angle_batch < 0 || c->angle_batch > RSX_MAX_ANGLE_BATCH)
    return fail(RSX_ERR_INVALID, "angle_batch=%d outside [0, %d]", c->angle_batch,
                RSX_MAX_ANGLE_BATCH);
  return RSX_OK;
}

size_t complex_size(int precision) { return precision == 32 ? 8 : 16; }
size_t real_size(int precision) { return precision == 32 ? 4 : 8; }
size_t geo_size(int precision) {
  return precision == 32 ? sizeof(Geo<float>) : sizeof(Geo<double>);
}

}  // namespace

namespace rsx {
// Lets other translation units of the library report through rsx_last_error.
void set_last_error(const char* msg) { g_err = msg; }

int check_device_pointer(const void* p, int dev, const char* what) {
  if (!p) return fail(RSX_ERR_INVALID, "%s is NULL", what);
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error an unknown pointer leaves behind
    return fail(RSX_ERR_INVALID, "%s is not a CUDA device pointer", what);
  }
  if (at.type == cudaMemoryTypeManaged) return RSX_OK;
  if (at.type != cudaMemoryTypeDevice)
    return fail(RSX_ERR_INVALID, "%s is host memory, not device memory", what);
  if (at.device != dev)
    return fail(RSX_ERR_INVALID, "%s lives on device %d, the work runs on device %d", what,
                at.device, dev);
  return RSX_OK;
}
}  // namespace rsx

#define RSX_DEVPTR(ptr, dev, what)                                   \
  do {                                                               \
    const int rc_ = rsx::check_device_pointer((ptr), (dev), (what)); \
    if (rc_) return rc_;                                             \
  } while (0)

struct rsx_context {
  rsx_config cfg{};
  int dev = 0;
  long long N = 0, npix = 0;
  void* M_owned = nullptr;  // device copy of a host morphology
  const void* M = nullptr;  // morphology in use (owned or borrowed)
  void* dir = nullptr;      // FP64 Algorithm 1: the morphology's director, [c][3][N] double
  std::vector<double> energies, constants;
  void* p = nullptr;    // kx x 3 N complex workspace (one p per angle of a batch)
  int kx = 1;           // angle batch of the Algorithm 1 x pass
  void* img = nullptr;  // one detector image
  void* acc = nullptr;  // running sum of rotated images
  void* geo = nullptr;  // per-pixel Ewald geometry of energy geo_energy
  unsigned short* b0idx = nullptr;  // its lower q_z bins, packed (fused y+z passes)
  // Algorithm 2: N_t of energy nt_energy (5 complex per voxel); a host
  // morphology stays on the host and is streamed per component in chunks
  // through two staging buffers on a copy stream.
  void* nt = nullptr;
  int nt_energy = -1;
  const void* M_host = nullptr;
  void* stage[2] = {nullptr, nullptr};
  long long stage_vox = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
  // linearity fast path (algorithm 3): FFT'd N_t entries and their two q_z
  // bins per pixel for energy bins_energy
  void* ft = nullptr;
  void* bins5 = nullptr;
  int bins_energy = -1;
  int geo_energy = -1;
  void* twx = nullptr;
  void* twy = nullptr;
  void* twz = nullptr;
  void* tw4 = nullptr;  // four-step twiddles [k2][n1] for 1024-point axes
  void* tw2k = nullptr; // 2048-point rows: the four-step table, then W2048^n (n < 1024)
  // tensor maps of the p (3 fields) and, for algorithm 3, ft (5 fields)
  // buffers for the TMA y pass (FP32, ny = 1024); valid when the flag is set
  CUtensorMap tmap_p;
  CUtensorMap tmap_ft;
  CUtensorMap tmap_pz[RSX_MAX_ANGLE_BATCH];  // each angle's p for the fused y+z pass
  CUtensorMap tmap_ftz;  // ft (five N_t entries) for the fused y+z pass
  bool has_tmap_p = false, has_tmap_ft = false, has_tmap_pz = false, has_tmap_ftz = false;
  // bins of the fused y-FFT + pruned z pass (FP32, Algorithms 1 and 2):
  // [kYzSlots][nf][ny][nx] float4
  void* part = nullptr;
  // linearity path: the images of a batch of angles ([kMaxAngleBatch][ny][nx])
  void* imgs = nullptr;
  // page-locked staging of host output (grown on demand)
  void* host_stage = nullptr;
  size_t host_stage_bytes = 0;
  int n_sm = 0;
  unsigned wait_polls = rsx::kWaitPolls;  // bound of the pipelined kernels' waits
  int* flag = nullptr;
  int* err = nullptr;  // set by a kernel whose bounded wait timed out
  // per-phase timing: event pairs recorded around launches while enabled
  bool timing = false;
  struct Rec {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
};

namespace {

void free_all(rsx_context* c) {
  void* ptrs[] = {c->M_owned, c->p,    c->img, c->acc,  c->geo,  c->twx, c->twy,
                  c->twz,     c->tw4,  c->flag, c->err, c->part, c->imgs, c->dir, c->tw2k,
                  c->b0idx};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  c->recs.clear();
  c->pool.clear();
  for (int b = 0; b < 2; ++b) {
    if (c->stage[b]) cudaFree(c->stage[b]);
    if (c->ev_copied[b]) cudaEventDestroy(c->ev_copied[b]);
    if (c->ev_used[b]) cudaEventDestroy(c->ev_used[b]);
  }
  if (c->nt) cudaFree(c->nt);
  if (c->ft) cudaFree(c->ft);
  if (c->bins5) cudaFree(c->bins5);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->host_stage) cudaFreeHost(c->host_stage);
}

cudaEvent_t take_event(rsx_context* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Brackets one kernel launch with events when timing is on.
struct PhaseTimer {
  rsx_context* c;
  cudaStream_t s;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseTimer(rsx_context* c_, int phase_, cudaStream_t s_) : c(c_), s(s_), phase(phase_) {
    if (c->timing && (a = take_event(c))) cudaEventRecord(a, s);
  }
  ~PhaseTimer() {
    if (!a) return;
    cudaEvent_t b = take_event(c);
    if (!b) {
      c->pool.push_back(a);
      return;
    }
    cudaEventRecord(b, s);
    c->recs.push_back({phase, a, b});
  }
};

// Four-step twiddles tw4[k2 * 32 + n1] = exp(-2 pi i n1 k2 / 1024).
int upload_tw4(rsx_context* c) {
  const int prec = c->cfg.precision;
  std::vector<double> tw(2 * 1024);
  for (int k2 = 0; k2 < 32; ++k2)
    for (int n1 = 0; n1 < 32; ++n1) {
      const double a = -2.0 * kPi * (double)(n1 * k2) / 1024.0;
      tw[2 * (k2 * 32 + n1)] = cos(a);
      tw[2 * (k2 * 32 + n1) + 1] = sin(a);
    }
  RSX_CK(cudaMalloc(&c->tw4, complex_size(prec) * 1024), "twiddle table");
  if (prec == 64) {
    RSX_CK(cudaMemcpy(c->tw4, tw.data(), 16 * 1024, cudaMemcpyHostToDevice), "twiddle upload");
  } else {
    std::vector<float> f(tw.begin(), tw.end());
    RSX_CK(cudaMemcpy(c->tw4, f.data(), 8 * 1024, cudaMemcpyHostToDevice), "twiddle upload");
  }
  return RSX_OK;
}

// Twiddles of the 2048-point row transform (FP32): the four-step table
// W1024^(n1 k2) at [k2 * 32 + n1], then W2048^n for n < 1024.
int upload_tw2k(rsx_context* c) {
  std::vector<float> tw(2 * 2048);
  for (int k2 = 0; k2 < 32; ++k2)
    for (int n1 = 0; n1 < 32; ++n1) {
      const double a = -2.0 * kPi * (double)(n1 * k2) / 1024.0;
      tw[2 * (k2 * 32 + n1)] = (float)cos(a);
      tw[2 * (k2 * 32 + n1) + 1] = (float)sin(a);
    }
  for (int n = 0; n < 1024; ++n) {
    const double a = -2.0 * kPi * (double)n / 2048.0;
    tw[2 * (1024 + n)] = (float)cos(a);
    tw[2 * (1024 + n) + 1] = (float)sin(a);
  }
  RSX_CK(cudaMalloc(&c->tw2k, 8 * 2048), "twiddle table");
  RSX_CK(cudaMemcpy(c->tw2k, tw.data(), 8 * 2048, cudaMemcpyHostToDevice), "twiddle upload");
  return RSX_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return nullptr;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  return encode;
}

// A tensor map over `nslices` [ny][nx] complex float planes (fields x
// z-slices, or fields x kept q_z planes) viewed as [nslices][ny][2 nx]
// floats with box_x x 256 x 1 boxes (box_x floats: 16 for 8-column tiles,
// 32 for 16-column tiles).
bool make_tmap(rsx_context* c, void* base, long long nslices, CUtensorMap* m, unsigned box_x,
               CUtensorMapL2promotion promo) {
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tmap_encoder();
  if (!encode) return false;
  const rsx_config& g = c->cfg;
  const cuuint64_t dims[3] = {2 * (cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)nslices};
  const cuuint64_t strides[2] = {2 * (cuuint64_t)g.nx * sizeof(float),
                                 (cuuint64_t)g.ny * 2 * g.nx * sizeof(float)};
  const cuuint32_t box[3] = {box_x, 256, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// The z-first pass's tensor map over the FP32 morphology, viewed as
// [c nz][ny][4 nx] floats: boxes of 128 / nz adjacent voxels (4 floats each)
// of one row y by the nz slices of one component (16 KB).
bool make_tmap_m(rsx_context* c, CUtensorMap* m) {
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tmap_encoder();
  if (!encode || !c->M || ((uintptr_t)c->M & 15)) return false;
  const rsx_config& g = c->cfg;
  const cuuint64_t dims[3] = {4 * (cuuint64_t)g.nx, (cuuint64_t)g.ny,
                              (cuuint64_t)g.n_components * g.nz};
  const cuuint64_t strides[2] = {4 * (cuuint64_t)g.nx * sizeof(float),
                                 (cuuint64_t)g.ny * 4 * g.nx * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)(4 * (1024 / g.nz)), 1, (cuuint32_t)g.nz};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(c->M), dims, strides, box,
                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// y-FFT of nbatch = k * nz (component, slice) batches: the TMA four-step
// kernel for FP32 with ny = 1024 (when its tensor map exists), the four-step
// kernel for ny = 1024, the Stockham column kernel otherwise.
template <typename R>
cudaError_t launch_y_fft(rsx_context* c, void* data, long long ncomp, cudaStream_t s) {
  const rsx_config& g = c->cfg;
  const rsx::ColBatches bt = {ncomp * g.nz, g.nz, c->N, c->npix, 0};
  const CUtensorMap* tm = data == c->p && c->has_tmap_p     ? &c->tmap_p
                          : data == c->ft && c->has_tmap_ft ? &c->tmap_ft
                                                             : nullptr;
  if (sizeof(R) == 4 && tm)
    return rsx::launch_col_fft4s_tma(tm, data, g.nx, g.nx, bt, c->tw4, c->err, c->n_sm,
                                     c->wait_polls, s);
  if (g.ny == 1024 && g.nx % 8 == 0 && c->tw4)
    return rsx::launch_col_fft4s<R>(data, g.nx, g.nx, bt, c->tw4, s);
  return rsx::launch_col_fft<R>(data, g.ny, g.nx, g.nx, bt, c->twy, s);
}

// exp(-2 pi i t / n), t < n, in the context precision.
int upload_twiddles(rsx_context* c, int n, void** dst) {
  const int prec = c->cfg.precision;
  std::vector<double> tw(2 * (size_t)n);
  for (int t = 0; t < n; ++t) {
    const double a = -2.0 * kPi * (double)t / (double)n;
    tw[2 * t] = cos(a);
    tw[2 * t + 1] = sin(a);
  }
  RSX_CK(cudaMalloc(dst, complex_size(prec) * n), "twiddle table");
  if (prec == 64) {
    RSX_CK(cudaMemcpy(*dst, tw.data(), 16 * (size_t)n, cudaMemcpyHostToDevice), "twiddle upload");
  } else {
    std::vector<float> f(tw.begin(), tw.end());
    RSX_CK(cudaMemcpy(*dst, f.data(), 8 * (size_t)n, cudaMemcpyHostToDevice), "twiddle upload");
  }
  return RSX_OK;
}

template <typename R>
PolParams<R> make_params(const rsx_context* c, int ie, double alpha, int add_ref) {
  PolParams<R> pp;
  memset(&pp, 0, sizeof(pp));
  const int nc = c->cfg.n_components;
  const double* k = c->constants.data() + (size_t)ie * nc * 4;
  for (int j = 0; j < nc; ++j) {
    // eps = n - 1 = -delta + i beta (Sec. 3.2)
    const double epr = -k[4 * j], epi = k[4 * j + 1];
    const double eqr = -k[4 * j + 2], eqi = k[4 * j + 3];
    const double tr = (epr + 2.0 * eqr) / 3.0, ti = (epi + 2.0 * eqi) / 3.0;
    rsx::set_component(pp, j, tr, ti, eqr - tr, eqi - ti, epr - eqr, epi - eqi);
  }
  pp.ce = (R)cos(alpha);
  pp.se = (R)sin(alpha);
  pp.c = nc;
  pp.literal = c->cfg.frame == RSX_FRAME_LITERAL;
  pp.add_ref = add_ref;
  return pp;
}

double wavenumber(double E) { return 2.0 * kPi / (kHcEvNm / E); }

template <typename R>
int ensure_geo(rsx_context* c, int ie, cudaStream_t s) {
  if (c->geo_energy == ie) return RSX_OK;
  PhaseTimer pt(c, RSX_PHASE_OTHER, s);
  RSX_CK(rsx::launch_geometry<R>((Geo<R>*)c->geo, c->cfg.nx, c->cfg.ny, c->cfg.nz,
                                 c->cfg.voxel_nm, wavenumber(c->energies[ie]), s, c->b0idx),
         "geometry kernel");
  c->geo_energy = ie;
  return RSX_OK;
}

// Algorithm 3 for energy ie into c->nt (once per energy): from the
// device-resident morphology in one pass, or streamed from the host one
// component at a time in chunks of stage_vox voxels, the copy of chunk i + 1
// (copy stream) overlapping the accumulation of chunk i (stream s).
template <typename R>
int ensure_nt(rsx_context* c, int ie, cudaStream_t s) {
  if (c->nt_energy == ie) return RSX_OK;
  const PolParams<R> pp = make_params<R>(c, ie, 0.0, 0);
  PhaseTimer pt(c, RSX_PHASE_NT, s);
  if (!c->M_host) {
    RSX_CK(rsx::launch_nt_all<R>(c->M, c->N, pp, c->nt, s), "N_t kernel");
    c->nt_energy = ie;
    return RSX_OK;
  }
  const size_t entry = 4 * sizeof(R);
  const long long N = c->N, CH = c->stage_vox;
  const long long nchunk = (N + CH - 1) / CH;
  // the copy stream starts after everything already queued on s
  RSX_CK(cudaEventRecord(c->ev_used[0], s), "N_t stream");
  RSX_CK(cudaEventRecord(c->ev_used[1], s), "N_t stream");
  long long step = 0;
  for (int j = 0; j < c->cfg.n_components; ++j) {
    for (long long ch = 0; ch < nchunk; ++ch, ++step) {
      const int b = (int)(step & 1);
      const long long off = ch * CH, n = (off + CH <= N) ? CH : N - off;
      const char* src = (const char*)c->M_host + ((size_t)j * N + off) * entry;
      RSX_CK(cudaStreamWaitEvent(c->copy_stream, c->ev_used[b], 0), "N_t stream");
      RSX_CK(cudaMemcpyAsync(c->stage[b], src, (size_t)n * entry, cudaMemcpyHostToDevice,
                             c->copy_stream),
             "morphology stream");
      RSX_CK(cudaEventRecord(c->ev_copied[b], c->copy_stream), "N_t stream");
      RSX_CK(cudaStreamWaitEvent(s, c->ev_copied[b], 0), "N_t stream");
      RSX_CK(rsx::launch_nt_comp<R>(c->stage[b], off, n, N, j, j == 0, pp, c->nt, s),
             "N_t kernel");
      RSX_CK(cudaEventRecord(c->ev_used[b], s), "N_t stream");
    }
  }
  c->nt_energy = ie;
  return RSX_OK;
}

// The fused y-FFT + q_z bins pass over nf fields (3: p; 5: the linearity
// path's N_t entries) through the tensor map `map`: the 1024-row kernel or
// the 512-row one.
// sel: the z-first path's ns planes per field (sel.nzfull > 0) instead of
// the nz slices.
cudaError_t fused_yz(rsx_context* c, const CUtensorMap* map, int nf, long long* L, cudaStream_t s,
                     rsx::YzSel sel = rsx::YzSel(), int ns = 0) {
  const rsx_config& g = c->cfg;
  const int nzv = sel.nzfull > 0 ? ns : g.nz;
  if (g.ny == 512)
    return rsx::launch_yz512_tma(map, g.nx, nzv, nf, (const Geo<float>*)c->geo, c->twz, c->twy,
                                 c->b0idx, c->part, c->err, c->n_sm, c->wait_polls, L, s, sel);
  return rsx::launch_yz_tma(map, g.nx, g.ny, nzv, nf, (const Geo<float>*)c->geo, c->twz, c->tw4,
                            g.ny == 2048 ? c->twy : nullptr, c->b0idx, c->part, c->err, c->n_sm,
                            c->wait_polls, L, s, sel);
}

// Linearity fast path, once per energy: FFT (x and y) of N_t's five
// entries, then their two q_z bins per pixel.
template <typename R>
int ensure_bins(rsx_context* c, int ie, cudaStream_t s) {
  if (c->bins_energy == ie) return RSX_OK;
  const rsx_config& g = c->cfg;
  int rc = ensure_geo<R>(c, ie, s);
  if (rc) return rc;
  if ((rc = ensure_nt<R>(c, ie, s))) return rc;
  {
    PhaseTimer pt(c, RSX_PHASE_POL_FFTX, s);
    RSX_CK(g.nx == 1024 && c->tw4
               ? rsx::launch_row_fft4s<R>(c->ft, 5LL * g.ny * g.nz, c->tw4, s, c->nt)
               : rsx::launch_row_fft<R>(c->ft, g.nx, 5LL * g.ny * g.nz, c->twx, s, c->nt),
           "x-FFT kernel");
  }
  const double dc = -(double)(g.n_components - 1) / (4.0 * kPi) * (double)c->N;
  if constexpr (sizeof(R) == 4) {
    if (c->part && c->has_tmap_ftz) {  // y-FFT and the q_z bins in one pass
      long long L = 0;
      {
        PhaseTimer pt(c, RSX_PHASE_FFTY, s);
        RSX_CK(fused_yz(c, &c->tmap_ftz, 5, &L, s), "y-FFT + z-bins kernel");
      }
      PhaseTimer pt(c, RSX_PHASE_EWALD, s);
      RSX_CK(rsx::launch_bins5_from_part(c->part, g.nx, g.ny, g.nz, L, (const Geo<float>*)c->geo,
                                         (float)dc, c->bins5, s),
             "q_z bins kernel");
      c->bins_energy = ie;
      return RSX_OK;
    }
  }
  if (g.ny > 1) {
    PhaseTimer pt(c, RSX_PHASE_FFTY, s);
    RSX_CK(launch_y_fft<R>(c, c->ft, 5, s), "y-FFT kernel");
  }
  PhaseTimer pt(c, RSX_PHASE_EWALD, s);
  RSX_CK(rsx::launch_zbins5<R>(c->ft, g.nx, g.ny, g.nz, (const Geo<R>*)c->geo, c->twz, dc,
                               c->bins5, s),
         "q_z bins kernel");
  c->bins_energy = ie;
  return RSX_OK;
}

// The x pass (polarisation fused with the x-FFT) into c->p: the bulk-copy
// pipelines for FP32 with nx = 1024 or 512 (morphology or N_t), the
// four-step kernel with plain loads for other nx = 1024 cases, the Stockham
// kernels for other sizes.
template <typename R>
int x_pass(rsx_context* c, const PolParams<R>& pp, cudaStream_t s) {
  const rsx_config& g = c->cfg;
  PhaseTimer pt(c, RSX_PHASE_POL_FFTX, s);
  if constexpr (sizeof(R) == 4) {
    const bool fast = (g.nx == 1024 || g.nx == 512) && c->n_sm > 0;
    const void* tw = g.nx == 1024 ? c->tw4 : c->twx;
    if (fast && g.algorithm == 1 && ((uintptr_t)c->M & 15) == 0) {
      RSX_CK(rsx::launch_pol_fft4s_tma(c->M, g.nx, g.ny, g.nz, pp, c->p, tw, c->err, c->n_sm,
                                       c->wait_polls, s),
             "polarisation + x-FFT kernel");
      return RSX_OK;
    }
    if (fast && g.algorithm == 2) {
      RSX_CK(rsx::launch_ntp_fft4s_tma(c->nt, g.nx, g.ny, g.nz, pp, c->p, tw, c->err, c->n_sm,
                                       c->wait_polls, s),
             "N_t polarisation + x-FFT kernel");
      return RSX_OK;
    }
  }
  if (g.nx == 1024) {
    RSX_CK(rsx::launch_pol_fft4s<R>(c->M, g.algorithm == 2 ? c->nt : nullptr, g.nx, g.ny, g.nz, pp,
                                    c->p, c->tw4, s, g.algorithm == 1 ? c->dir : nullptr),
           "polarisation + x-FFT kernel");
  } else if (g.algorithm == 2) {
    RSX_CK(rsx::launch_ntp_fftx<R>(c->nt, g.nx, g.ny, g.nz, pp, true, c->p, c->twx, s),
           "N_t polarisation + x-FFT kernel");
  } else {
    RSX_CK(rsx::launch_pol_fftx<R>(c->M, g.nx, g.ny, g.nz, pp, true, c->p, c->twx, s, 0, -1,
                                   c->dir),
           "polarisation + x-FFT kernel");
  }
  return RSX_OK;
}

template <typename R>
int scatter_angle(rsx_context* c, int ie, double alpha, void* img, cudaStream_t s) {
  const rsx_config& g = c->cfg;
  int rc = ensure_geo<R>(c, ie, s);
  if (rc) return rc;
  if (g.algorithm == 3) {
    if ((rc = ensure_bins<R>(c, ie, s))) return rc;
    PhaseTimer pt(c, RSX_PHASE_EWALD, s);
    RSX_CK(rsx::launch_ewald_linear<R>(c->bins5, g.nx, g.ny, (const Geo<R>*)c->geo, alpha,
                                       g.frame == RSX_FRAME_LITERAL, img, s),
           "Ewald kernel");
    return RSX_OK;
  }
  if (g.algorithm == 2 && (rc = ensure_nt<R>(c, ie, s))) return rc;
  if ((rc = x_pass<R>(c, make_params<R>(c, ie, alpha, 0), s))) return rc;
  // The constant -(c-1) e' / (4 pi) left out of p before the FFT returns at
  // q = 0 as N times itself (e' = x-hat in the literal frame, e otherwise).
  const double ref = -(double)(g.n_components - 1) / (4.0 * kPi) * (double)c->N;
  R dc[3];
  if (g.frame == RSX_FRAME_LITERAL) {
    dc[0] = (R)ref; dc[1] = (R)0; dc[2] = (R)0;
  } else {
    dc[0] = (R)(ref * cos(alpha)); dc[1] = (R)(ref * sin(alpha)); dc[2] = (R)0;
  }
  if constexpr (sizeof(R) == 4) {
    if (c->part && c->has_tmap_pz) {  // y-FFT and the pruned z transform in one pass
      long long L = 0;
      {
        PhaseTimer pt(c, RSX_PHASE_FFTY, s);
        RSX_CK(fused_yz(c, &c->tmap_pz[0], 3, &L, s), "y-FFT + z-bins kernel");
      }
      PhaseTimer pt(c, RSX_PHASE_EWALD, s);
      RSX_CK(rsx::launch_ewald_bins(c->part, g.nx, g.ny, g.nz, L, (const Geo<float>*)c->geo,
                                    dc[0], dc[1], dc[2], (float*)img, s),
             "Ewald kernel");
      return RSX_OK;
    }
  }
  if (g.ny > 1) {
    PhaseTimer pt(c, RSX_PHASE_FFTY, s);
    RSX_CK(launch_y_fft<R>(c, c->p, 3, s), "y-FFT kernel");
  }
  PhaseTimer pt(c, RSX_PHASE_EWALD, s);
  RSX_CK(rsx::launch_ewald<R>(c->p, g.nx, g.ny, g.nz, (const Geo<R>*)c->geo, c->twz, true, dc, img,
                              s, c->err, c->wait_polls),
         "Ewald kernel");
  return RSX_OK;
}

int check_ready(const rsx_context* c) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  if (!c->M) return fail(RSX_ERR_STATE, "morphology not set");
  if (c->energies.empty()) return fail(RSX_ERR_STATE, "optical constants not set");
  return RSX_OK;
}

int check_energy(const rsx_context* c, int ie) {
  if (ie < 0 || ie >= (int)c->energies.size())
    return fail(RSX_ERR_INVALID, "energy index %d outside [0, %d)", ie, (int)c->energies.size());
  return RSX_OK;
}

// Reads and clears the kernel error flag (the caller has synchronised the
// work it covers).  When it was set, per-energy data an aborted kernel may
// have produced is dropped and RSX_ERR_CUDA returned.
int take_kernel_error(rsx_context* c) {
  int h = 0;
  RSX_CK(cudaMemcpy(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost), "kernel error flag");
  if (!h) return RSX_OK;
  RSX_CK(cudaMemset(c->err, 0, sizeof(int)), "kernel error flag");
  c->nt_energy = -1;
  c->bins_energy = -1;
  c->geo_energy = -1;
  return fail(RSX_ERR_CUDA, "a kernel pipeline wait timed out; the result is not valid");
}

bool host_morphology_ok(const void* M, int prec, long long n) {
  for (long long i = 0; i < n; ++i) {
    double v, s, ph, th;
    if (prec == 32) {
      const float* f = (const float*)M + 4 * i;
      v = f[0]; s = f[1]; ph = f[2]; th = f[3];
    } else {
      const double* d = (const double*)M + 4 * i;
      v = d[0]; s = d[1]; ph = d[2]; th = d[3];
    }
    if (!(v >= 0.0 && v <= 1.0 && s >= 0.0 && s <= 1.0 && isfinite(ph) && isfinite(th)))
      return false;
  }
  return true;
}

}  // namespace

// ======================================================================= ABI
// Every function below is declared extern "C" in rsx.h and keeps that linkage.

const char* rsx_last_error(void) { return g_err.c_str(); }

// The fused y-FFT + pruned z pass serves FP32 Algorithms 1 and 2 on
// qualifying shapes; its bins take 2 x 3 x 16 bytes per pixel.
static bool uses_yz(const rsx_config* cfg) {
  return cfg->precision == 32 && rsx::yz_fusable(cfg->nx, cfg->ny, cfg->nz);
}
// kYzSlots slots of (3 fields of p, or the linearity path's 5 N_t entries) x 2 bins
static size_t part_bytes(const rsx_config* cfg) {
  return rsx::kYzSlots * (size_t)(cfg->algorithm == 3 ? 5 : 3) * cfg->nx * cfg->ny * 16;
}

// The z-first path serves FP32 Algorithm 1 with nz = 32, 64 or 128 and
// nx, ny = 512, 1024 or 2048.
static bool zfirst_ok(const rsx_config* cfg) {
  return cfg->precision == 32 && cfg->algorithm == 1 &&
         rsx::zfirst_fusable(cfg->nx, cfg->ny, cfg->nz);
}

// The multi-angle x pass serves FP32 Algorithm 1 with nx = 512, 1024 or
// 2048 (2048-point rows: at most 3 angles per pass).
static int x_multi_cap(const rsx_config* cfg) {
  if (cfg->precision != 32 || cfg->algorithm != 1) return 0;
  if (cfg->nx == 512 || cfg->nx == 1024) return RSX_MAX_ANGLE_BATCH;
  return cfg->nx == 2048 ? 3 : 0;
}

// The angle batch a config gets (the number of p buffers): up to 8 where
// the z-first path or the multi-angle x pass serves it.
static int angle_batch_cap(const rsx_config* cfg) {
  return zfirst_ok(cfg) ? RSX_MAX_ANGLE_BATCH : x_multi_cap(cfg);
}

static int angle_batch_of(const rsx_config* cfg) {
  const int cap = angle_batch_cap(cfg);
  if (cap == 0) return 1;
  if (cfg->angle_batch > 0) return cfg->angle_batch < cap ? cfg->angle_batch : cap;
  // default: the largest batch up to the cap whose p buffers (3 N complex
  // float each) fit in 32 GiB
  const double p_bytes = 3.0 * cfg->nx * cfg->ny * cfg->nz * 8.0;
  const int k = (int)((double)(32LL << 30) / p_bytes);
  return k < 1 ? 1 : k > cap ? cap : k;
}

// The z-first path's plan for one energy: the cyclic run of q_z bins its
// pixels read and the angles per pass.  The run ends at bin 1 (q_z <= 0
// on the sphere, so b0 <= 0, b1 <= 1) and starts at the lowest b0 =
// floor(t) over the pixels on the sphere (Eq. (Ewald) in double, as
// k_geometry evaluates it), reached per row at the largest |q_x| still on
// the sphere.  The device rounds in another order, so the bound is taken
// wide enough for any such difference: a pixel within 1e-12 k^2 of the
// sphere's edge counts as on it (at q_z = -k, its lowest possible value),
// and a t within 1e-9 above an integer also takes the bin below.
struct ZPlan {
  int kb = 0, ns = 0, kz = 0;
};

static int lowest_bin(const rsx_config& g, double k) {
  const double two_pi = 2.0 * kPi;
  const double dqx = two_pi / (g.nx * g.voxel_nm), dqz = two_pi / (g.nz * g.voxel_nm);
  const double edge = 1e-12 * k * k;
  const int fmax = g.nx / 2;  // largest |f_x| on the FFT grid (nx even)
  double tmin = 0.0;
  for (int my = 0; my < g.ny; ++my) {
    const int fy = my < (g.ny + 1) / 2 ? my : my - g.ny;
    const double qy = two_pi * fy / (g.ny * g.voxel_nm);
    const double r2 = k * k - qy * qy + edge;
    if (r2 < 0.0) continue;
    const double fl = floor(sqrt(r2) / dqx);
    int f = fl < (double)fmax ? (int)fl : fmax;
    while (f < fmax && (dqx * (f + 1)) * (dqx * (f + 1)) <= r2) ++f;
    while (f > 0 && (dqx * f) * (dqx * f) > r2) --f;
    const double qx = dqx * f;
    const double rad = k * k - qx * qx - qy * qy;
    if (rad < -edge) continue;
    const double t = (-k + sqrt(rad > 0.0 ? rad : 0.0)) / dqz;
    if (t < tmin) tmin = t;
  }
  double lo = floor(tmin);
  if (tmin - lo < 1e-9 * (1.0 + fabs(tmin))) lo -= 1.0;
  return (int)lo;
}

// The plan from the shape, the angle batch kx (p buffers of 3 nz planes
// each) and the wavenumber k alone (host arithmetic, no device state).
static bool zfirst_plan_of(const rsx_config& g, int kx, double k, ZPlan* zp) {
  if (!zfirst_ok(&g)) return false;
  const int blo = lowest_bin(g, k);
  const int ns = 2 - blo;
  // worth it while at most 3/4 of the bins are kept (the z transform costs
  // about what the dropped planes' x and y transforms save at ~0.8)
  if (4 * ns > 3 * g.nz) return false;
  zp->ns = ns;
  zp->kb = ((blo % g.nz) + g.nz) % g.nz;
  // the kept planes of kz angles fit in the kx p buffers of 3 nz planes each
  const int kz = (int)((long long)kx * g.nz / ns);
  zp->kz = kz < rsx::kMaxXAngles ? kz : rsx::kMaxXAngles;
  return zp->kz >= 1;
}

static bool zfirst_plan(const rsx_context* c, int ie, ZPlan* zp) {
  const rsx_config& g = c->cfg;
  if (!zfirst_ok(&g) || c->n_sm <= 0 || !c->part || !c->b0idx || ie < 0 ||
      ie >= (int)c->energies.size() || (c->M && ((uintptr_t)c->M & 15)))
    return false;
  if ((g.nx == 1024 && !c->tw4) || (g.nx == 2048 && !c->tw2k) || (g.ny == 2048 && !c->twy))
    return false;
  return zfirst_plan_of(g, c->kx, wavenumber(c->energies[ie]), zp);
}

size_t rsx_workspace_bytes(const rsx_config* cfg) {
  if (check_config(cfg) != RSX_OK) return 0;
  const long long N = (long long)cfg->nx * cfg->ny * cfg->nz;
  const long long npix = (long long)cfg->nx * cfg->ny;
  const size_t R = real_size(cfg->precision), Cs = complex_size(cfg->precision);
  const long long stage_vox = N < (1LL << 22) ? N : (1LL << 22);
  size_t b = cfg->algorithm == 1
                 ? (size_t)cfg->n_components * N * 4 * R  // morphology copy (Table 1: 4c N)
                 : 5 * (size_t)N * Cs + 2 * (size_t)stage_vox * 4 * R;  // N_t + staging (Table 2)
  if (cfg->algorithm == 3) b += 5 * (size_t)N * Cs + 10 * (size_t)npix * Cs;  // FFT'd N_t, bins
  b += 3 * (size_t)N * Cs * angle_batch_of(cfg);     // p_x, p_y, p_z (Table 1: 6 N) per angle
  if (cfg->precision == 64 && cfg->algorithm == 1)
    b += 3 * (size_t)cfg->n_components * N * R;      // the cached director
  b += 2 * (size_t)npix * R;                         // Ewald, Ewald_Avg (Table 1: 2 nx ny)
  b += (size_t)npix * geo_size(cfg->precision);
  b += (size_t)(cfg->nx + cfg->ny + cfg->nz) * Cs + sizeof(int);
  if (uses_yz(cfg)) b += part_bytes(cfg) + 2 * (size_t)npix;  // fused y + z pass: bins, bin indices
  if (cfg->algorithm == 3) b += (size_t)rsx::kMaxAngleBatch * npix * R;  // a batch of images
  return b;
}

int rsx_angle_batch(const rsx_context* c) { return c ? c->kx : -1; }

int rsx_zfirst_plan(const rsx_context* c, int ie, int* n_planes, int* first_bin,
                    int* angles_per_pass) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  if (c->energies.empty()) return fail(RSX_ERR_STATE, "no optical constants set");
  if (ie < 0 || ie >= (int)c->energies.size())
    return fail(RSX_ERR_INVALID, "energy index %d out of range [0, %zu)", ie, c->energies.size());
  ZPlan zp;
  if (!zfirst_plan(c, ie, &zp)) zp = ZPlan();
  if (n_planes) *n_planes = zp.ns;
  if (first_bin) *first_bin = zp.kb;
  if (angles_per_pass) *angles_per_pass = zp.kz;
  return RSX_OK;
}

int rsx_zfirst_plan_for(const rsx_config* cfg, double energy_ev, int* n_planes, int* first_bin,
                        int* angles_per_pass) {
  const int rc = check_config(cfg);
  if (rc) return rc;
  if (!isfinite(energy_ev) || !(energy_ev > 0.0))
    return fail(RSX_ERR_INVALID, "energy must be finite and > 0 (got %g eV)", energy_ev);
  ZPlan zp;
  if (!zfirst_plan_of(*cfg, angle_batch_of(cfg), wavenumber(energy_ev), &zp)) zp = ZPlan();
  if (n_planes) *n_planes = zp.ns;
  if (first_bin) *first_bin = zp.kb;
  if (angles_per_pass) *angles_per_pass = zp.kz;
  return RSX_OK;
}

int rsx_angle_count(double start, double inc, double end, int rotation) {
  if (!rotation) return 1;
  if (!isfinite(start) || !isfinite(inc) || !isfinite(end) || !(inc > 0.0) || end < start)
    return -1;
  const double n = floor((end - start) / inc + 1e-6) + 1.0;
  if (n > 1e7) return -1;
  return (int)n;
}

int rsx_create(const rsx_config* cfg, rsx_context** out) {
  if (!out) return fail(RSX_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int rc = check_config(cfg);
  if (rc) return rc;
  rsx_context* c = new (std::nothrow) rsx_context();
  if (!c) return fail(RSX_ERR_OOM, "no host memory for the context");
  c->cfg = *cfg;
  c->N = (long long)cfg->nx * cfg->ny * cfg->nz;
  c->npix = (long long)cfg->nx * cfg->ny;
  c->kx = angle_batch_of(cfg);
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaGetDevice");
  }
  const size_t R = real_size(cfg->precision), Cs = complex_size(cfg->precision);
  struct {
    void** dst;
    size_t bytes;
    const char* what;
  } allocs[] = {
      {&c->p, 3 * (size_t)c->N * Cs * c->kx, "p workspace"},
      {&c->img, (size_t)c->npix * R, "Ewald image"},
      {&c->acc, (size_t)c->npix * R, "Ewald average"},
      {&c->geo, (size_t)c->npix * geo_size(cfg->precision), "Ewald geometry"},
      {(void**)&c->flag, sizeof(int), "validation flag"},
      {(void**)&c->err, sizeof(int), "kernel error flag"},
  };
  for (auto& a : allocs) {
    e = cudaMalloc(a.dst, a.bytes);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, a.what);
      free_all(c);
      delete c;
      return rc;
    }
  }
  if (cfg->algorithm >= 2) {
    c->stage_vox = c->N < (1LL << 22) ? c->N : (1LL << 22);
    e = cudaMalloc(&c->nt, 5 * (size_t)c->N * Cs);
    if (e == cudaSuccess && cfg->algorithm == 3) e = cudaMalloc(&c->ft, 5 * (size_t)c->N * Cs);
    if (e == cudaSuccess && cfg->algorithm == 3) e = cudaMalloc(&c->bins5, 10 * (size_t)c->npix * Cs);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaMalloc(&c->stage[b], (size_t)c->stage_vox * 4 * R);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_copied[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_used[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "Algorithm 2 buffers");
      free_all(c);
      delete c;
      return rc;
    }
  }
  if (cfg->precision == 64 && cfg->algorithm == 1 &&
      (e = cudaMalloc(&c->dir, 3 * (size_t)cfg->n_components * c->N * R)) != cudaSuccess) {
    rc = cuda_fail(e, "director cache");
    free_all(c);
    delete c;
    return rc;
  }
  e = cudaMemset(c->err, 0, sizeof(int));
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "kernel error flag");
    free_all(c);
    delete c;
    return rc;
  }
  if ((cfg->nx == 1024 || cfg->ny == 1024 || (cfg->ny == 2048 && uses_yz(cfg))) &&
      (rc = upload_tw4(c))) {
    free_all(c);
    delete c;
    return rc;
  }
  if (cfg->nx == 2048 && angle_batch_cap(cfg) && (rc = upload_tw2k(c))) {
    free_all(c);
    delete c;
    return rc;
  }
  if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess)
    c->n_sm = 0;
  if (cfg->precision == 32 && cfg->ny == 1024 && cfg->nx % 8 == 0 && c->n_sm > 0) {
    c->has_tmap_p =
        make_tmap(c, c->p, 3LL * cfg->nz, &c->tmap_p, 16, CU_TENSOR_MAP_L2_PROMOTION_L2_256B);
    if (c->ft)
      c->has_tmap_ft =
          make_tmap(c, c->ft, 5LL * cfg->nz, &c->tmap_ft, 16, CU_TENSOR_MAP_L2_PROMOTION_L2_256B);
  }
  if (uses_yz(cfg) && c->n_sm > 0) {
    // the fused y+z pass: 1024-row tiles are 8 columns wide and two blocks
    // read the halves of each 128-byte line at once, 2048-row tiles 4
    // columns (four blocks), 512-row tiles are 16 columns (whole lines);
    // promote to 128 bytes, not 256
    const unsigned box = cfg->ny == 512 ? 32 : cfg->ny == 2048 ? 8 : 16;
    c->has_tmap_pz = true;
    for (int k = 0; k < c->kx; ++k)
      c->has_tmap_pz = c->has_tmap_pz &&
                       make_tmap(c, (char*)c->p + (size_t)k * 3 * c->N * Cs, 3LL * cfg->nz,
                                 &c->tmap_pz[k], box, CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
    if (c->ft)
      c->has_tmap_ftz = make_tmap(c, c->ft, 5LL * cfg->nz, &c->tmap_ftz, box,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
  }
  if (cfg->algorithm == 3 &&
      (e = cudaMalloc(&c->imgs, (size_t)rsx::kMaxAngleBatch * c->npix * R)) != cudaSuccess) {
    rc = cuda_fail(e, "linearity path images");
    free_all(c);
    delete c;
    return rc;
  }
  if (uses_yz(cfg) && ((e = cudaMalloc(&c->part, part_bytes(cfg))) != cudaSuccess ||
                       (e = cudaMalloc((void**)&c->b0idx, (size_t)c->npix * 2)) != cudaSuccess)) {
    rc = cuda_fail(e, "y + z pass bins");
    free_all(c);
    delete c;
    return rc;
  }
  if ((rc = upload_twiddles(c, cfg->nx, &c->twx)) || (rc = upload_twiddles(c, cfg->ny, &c->twy)) ||
      (rc = upload_twiddles(c, cfg->nz, &c->twz))) {
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return RSX_OK;
}

int rsx_destroy(rsx_context* c) {
  if (!c) return RSX_OK;
  DeviceGuard dg(c->dev);
  free_all(c);
  delete c;
  return RSX_OK;
}

int rsx_set_morphology(rsx_context* c, const void* M, int where, void* stream) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  if (!M) return fail(RSX_ERR_INVALID, "morphology pointer is NULL");
  if (where != RSX_HOST && where != RSX_DEVICE && where != RSX_HOST_ASYNC)
    return fail(RSX_ERR_INVALID, "where=%d: must be RSX_HOST, RSX_DEVICE or RSX_HOST_ASYNC", where);
  DeviceGuard dg(c->dev);
  if (!dg.ok) return fail(RSX_ERR_CUDA, "cannot select the context's device");
  cudaStream_t s = (cudaStream_t)stream;
  const int prec = c->cfg.precision;
  const long long n_entries = (long long)c->cfg.n_components * c->N;
  const size_t bytes = (size_t)n_entries * 4 * real_size(prec);
  if (where == RSX_HOST_ASYNC && c->cfg.algorithm == 1) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, M) != cudaSuccess || at.type != cudaMemoryTypeHost) {
      cudaGetLastError();  // clear a sticky "invalid value" from an unknown pointer
      return fail(RSX_ERR_INVALID, "RSX_HOST_ASYNC needs page-locked host memory");
    }
  }
  if (where == RSX_HOST || where == RSX_HOST_ASYNC) {
    if (c->cfg.validate && !host_morphology_ok(M, prec, n_entries))
      return fail(RSX_ERR_INVALID, "morphology value outside 0<=v<=1, 0<=s<=1 or non-finite angle");
    if (c->cfg.algorithm >= 2) {
      // Algorithm 2 keeps the morphology on the host and streams it per
      // component for each energy (Algorithm 3): borrowed, not copied.
      c->M_host = M;
      c->M = M;
      c->nt_energy = -1;
      c->bins_energy = -1;
      return RSX_OK;
    }
    if (!c->M_owned) RSX_CK(cudaMalloc(&c->M_owned, bytes), "morphology copy");
    RSX_CK(cudaMemcpyAsync(c->M_owned, M, bytes, cudaMemcpyHostToDevice, s), "morphology upload");
    if (c->dir)
      RSX_CK(rsx::launch_director<double>(c->M_owned, n_entries, c->N, c->dir, s),
             "director kernel");
    if (where == RSX_HOST) RSX_CK(cudaStreamSynchronize(s), "morphology upload");
    c->M = c->M_owned;
    c->nt_energy = -1;
    c->bins_energy = -1;
    return RSX_OK;
  }
  RSX_DEVPTR(M, c->dev, "device morphology");
  if (((uintptr_t)M) % (4 * real_size(prec)) != 0)
    return fail(RSX_ERR_INVALID, "device morphology must be aligned to %d bytes",
                (int)(4 * real_size(prec)));
  if (c->cfg.validate) {
    int h = 0;
    RSX_CK(cudaMemsetAsync(c->flag, 0, sizeof(int), s), "validation");
    RSX_CK(prec == 32 ? rsx::launch_validate<float>(M, n_entries, c->flag, s)
                      : rsx::launch_validate<double>(M, n_entries, c->flag, s),
           "validation kernel");
    RSX_CK(cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, s), "validation");
    RSX_CK(cudaStreamSynchronize(s), "validation");
    if (h) return fail(RSX_ERR_INVALID, "morphology value outside 0<=v<=1, 0<=s<=1 or non-finite angle");
  }
  if (c->dir) {
    RSX_CK(rsx::launch_director<double>(M, n_entries, c->N, c->dir, s), "director kernel");
    RSX_CK(cudaStreamSynchronize(s), "director kernel");
  }
  c->M = M;
  c->M_host = nullptr;
  c->nt_energy = -1;
  c->bins_energy = -1;
  return RSX_OK;
}

int rsx_set_optical_constants(rsx_context* c, int n, const double* E, const double* k) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  if (n < 1 || !E || !k) return fail(RSX_ERR_INVALID, "need n_energies >= 1 and non-NULL arrays");
  const int nc = c->cfg.n_components;
  for (int i = 0; i < n; ++i)
    if (!(E[i] > 0.0) || !isfinite(E[i])) return fail(RSX_ERR_INVALID, "energy %d not positive", i);
  for (long long i = 0; i < (long long)n * nc * 4; ++i)
    if (!isfinite(k[i])) return fail(RSX_ERR_INVALID, "optical constant %lld not finite", i);
  c->energies.assign(E, E + n);
  c->constants.assign(k, k + (size_t)n * nc * 4);
  c->geo_energy = -1;
  c->nt_energy = -1;
  c->bins_energy = -1;
  return RSX_OK;
}

int rsx_polarization(rsx_context* c, int ie, double alpha, void* p_out, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_energy(c, ie))) return rc;
  if (!p_out) return fail(RSX_ERR_INVALID, "p_out is NULL");
  RSX_DEVPTR(p_out, c->dev, "p_out");
  DeviceGuard dg(c->dev);
  cudaStream_t s = (cudaStream_t)stream;
  const rsx_config& g = c->cfg;
  if (g.algorithm >= 2) {
    int rc2 = g.precision == 32 ? ensure_nt<float>(c, ie, s) : ensure_nt<double>(c, ie, s);
    if (rc2) return rc2;
    RSX_CK(g.precision == 32
               ? rsx::launch_ntp_fftx<float>(c->nt, g.nx, g.ny, g.nz,
                                             make_params<float>(c, ie, alpha, 1), false, p_out,
                                             nullptr, s)
               : rsx::launch_ntp_fftx<double>(c->nt, g.nx, g.ny, g.nz,
                                              make_params<double>(c, ie, alpha, 1), false, p_out,
                                              nullptr, s),
           "N_t polarisation kernel");
    return RSX_OK;
  }
  if (g.precision == 32) {
    RSX_CK(rsx::launch_pol_fftx<float>(c->M, g.nx, g.ny, g.nz, make_params<float>(c, ie, alpha, 1),
                                       false, p_out, nullptr, s),
           "polarisation kernel");
  } else {
    RSX_CK(rsx::launch_pol_fftx<double>(c->M, g.nx, g.ny, g.nz,
                                        make_params<double>(c, ie, alpha, 1), false, p_out, nullptr,
                                        s),
           "polarisation kernel");
  }
  return RSX_OK;
}

namespace {
template <typename R>
int fft3d_impl(rsx_context* c, void* p, cudaStream_t s) {
  const rsx_config& g = c->cfg;
  RSX_CK(g.nx == 1024 && c->tw4 ? rsx::launch_row_fft4s<R>(p, 3LL * g.ny * g.nz, c->tw4, s)
                                : rsx::launch_row_fft<R>(p, g.nx, 3LL * g.ny * g.nz, c->twx, s),
         "x-FFT kernel");
  RSX_CK(rsx::launch_col_fft<R>(p, g.ny, g.nx, g.nx, {3LL * g.nz, g.nz, c->N, c->npix, 0}, c->twy, s),
         "y-FFT kernel");
  if (g.nz == 1) return RSX_OK;
  if (g.nz <= 4096) {
    RSX_CK(rsx::launch_col_fft<R>(p, g.nz, c->npix, c->npix, {3, 1, c->N, 0, 0}, c->twz, s),
           "z-FFT kernel");
  } else {
    RSX_CK(rsx::launch_dft_z<R>(p, c->p, g.nx, g.ny, g.nz, c->twz, s), "z-DFT kernel");
    RSX_CK(cudaMemcpyAsync(p, c->p, 3 * (size_t)c->N * sizeof(R) * 2, cudaMemcpyDeviceToDevice, s),
           "z-DFT copy");
  }
  return RSX_OK;
}
}  // namespace

int rsx_fft3d(rsx_context* c, void* p, void* stream) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  if (!p) return fail(RSX_ERR_INVALID, "p is NULL");
  if (p == c->p) return fail(RSX_ERR_INVALID, "p must be a caller buffer");
  RSX_DEVPTR(p, c->dev, "p");
  DeviceGuard dg(c->dev);
  cudaStream_t s = (cudaStream_t)stream;
  return c->cfg.precision == 32 ? fft3d_impl<float>(c, p, s) : fft3d_impl<double>(c, p, s);
}

int rsx_ewald(rsx_context* c, int ie, const void* pt, void* img, void* stream) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  if (c->energies.empty()) return fail(RSX_ERR_STATE, "optical constants not set");
  int rc = check_energy(c, ie);
  if (rc) return rc;
  if (!pt || !img) return fail(RSX_ERR_INVALID, "NULL buffer");
  RSX_DEVPTR(pt, c->dev, "p_tilde");
  RSX_DEVPTR(img, c->dev, "img_out");
  DeviceGuard dg(c->dev);
  cudaStream_t s = (cudaStream_t)stream;
  const rsx_config& g = c->cfg;
  if (g.precision == 32) {
    if ((rc = ensure_geo<float>(c, ie, s))) return rc;
    const float dc[3] = {0, 0, 0};
    RSX_CK(rsx::launch_ewald<float>(pt, g.nx, g.ny, g.nz, (const Geo<float>*)c->geo, c->twz, false,
                                    dc, img, s),
           "Ewald kernel");
  } else {
    if ((rc = ensure_geo<double>(c, ie, s))) return rc;
    const double dc[3] = {0, 0, 0};
    RSX_CK(rsx::launch_ewald<double>(pt, g.nx, g.ny, g.nz, (const Geo<double>*)c->geo, c->twz,
                                     false, dc, img, s),
           "Ewald kernel");
  }
  return RSX_OK;
}

int rsx_rotate_accumulate(rsx_context* c, const void* img, double alpha, void* acc, void* stream) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  if (!img || !acc) return fail(RSX_ERR_INVALID, "NULL buffer");
  if (!isfinite(alpha)) return fail(RSX_ERR_INVALID, "alpha not finite");
  RSX_DEVPTR(img, c->dev, "img");
  RSX_DEVPTR(acc, c->dev, "acc");
  DeviceGuard dg(c->dev);
  cudaStream_t s = (cudaStream_t)stream;
  const rsx_config& g = c->cfg;
  RSX_CK(g.precision == 32 ? rsx::launch_rotate_acc<float>(img, acc, g.nx, g.ny, alpha, true, s)
                           : rsx::launch_rotate_acc<double>(img, acc, g.nx, g.ny, alpha, true, s),
         "rotation kernel");
  return RSX_OK;
}

int rsx_scatter_angle(rsx_context* c, int ie, double alpha, void* img, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_energy(c, ie))) return rc;
  if (!img) return fail(RSX_ERR_INVALID, "img_out is NULL");
  if (!isfinite(alpha)) return fail(RSX_ERR_INVALID, "alpha not finite");
  RSX_DEVPTR(img, c->dev, "img_out");
  DeviceGuard dg(c->dev);
  cudaStream_t s = (cudaStream_t)stream;
  return c->cfg.precision == 32 ? scatter_angle<float>(c, ie, alpha, img, s)
                                : scatter_angle<double>(c, ie, alpha, img, s);
}

namespace {
// All angles of one energy, one after the other: the image of each angle
// (scatter_angle), rotated into the average.
// Algorithm 1 with the morphology read once per batch of kx angles: the
// multi-angle x pass writes each angle's x-transformed p to its own buffer,
// then every angle of the batch goes through the fused y+z pass, the Ewald
// image and the rotation into the average, in angle order.
int run_energy_angles_batched(rsx_context* c, int ie, double start, double inc, int nang,
                              int rotation, cudaStream_t s) {
  const rsx_config& g = c->cfg;
  int rc = ensure_geo<float>(c, ie, s);
  if (rc) return rc;
  const PolParams<float> pp = make_params<float>(c, ie, 0.0, 0);
  const double ref = -(double)(g.n_components - 1) / (4.0 * kPi) * (double)c->N;
  const void* tw = g.nx == 1024 ? c->tw4 : g.nx == 2048 ? c->tw2k : c->twx;
  const bool fused = c->part && c->has_tmap_pz;
  const int cap = x_multi_cap(&g), kx = c->kx < cap ? c->kx : cap;
  for (int a0 = 0; a0 < nang; a0 += kx) {
    const int nk = nang - a0 < kx ? nang - a0 : kx;
    rsx::XAngles ang;
    memset(&ang, 0, sizeof(ang));
    ang.n = nk;
    double alpha[rsx::kMaxXAngles];
    for (int k = 0; k < nk; ++k) {
      alpha[k] = rotation ? (start + inc * (a0 + k)) * (kPi / 180.0) : 0.0;
      ang.ce[k] = (float)cos(alpha[k]);
      ang.se[k] = (float)sin(alpha[k]);
    }
    {
      PhaseTimer pt(c, RSX_PHASE_POL_FFTX, s);
      RSX_CK(rsx::launch_pol_fft4s_tma_multi(c->M, g.nx, g.ny, g.nz, pp, ang, c->p, 3 * c->N, tw,
                                             c->err, c->n_sm, c->wait_polls, s),
             "polarisation + x-FFT kernel");
    }
    for (int k = 0; k < nk; ++k) {
      float dc[3] = {(float)ref, 0.f, 0.f};
      if (g.frame != RSX_FRAME_LITERAL) {
        dc[0] = (float)(ref * cos(alpha[k]));
        dc[1] = (float)(ref * sin(alpha[k]));
      }
      if (fused) {  // y-FFT and the pruned z transform in one pass
        long long L = 0;
        {
          PhaseTimer pt(c, RSX_PHASE_FFTY, s);
          RSX_CK(fused_yz(c, &c->tmap_pz[k], 3, &L, s), "y-FFT + z-bins kernel");
        }
        PhaseTimer pt(c, RSX_PHASE_EWALD, s);
        RSX_CK(rsx::launch_ewald_bins(c->part, g.nx, g.ny, g.nz, L, (const Geo<float>*)c->geo,
                                      dc[0], dc[1], dc[2], (float*)c->img, s),
               "Ewald kernel");
      } else {  // y-FFT of angle k's p in place, then the pruned z transform
        void* pk = (char*)c->p + (size_t)k * 3 * c->N * sizeof(float2);
        if (g.ny > 1) {
          PhaseTimer pt(c, RSX_PHASE_FFTY, s);
          RSX_CK(launch_y_fft<float>(c, pk, 3, s), "y-FFT kernel");
        }
        PhaseTimer pt(c, RSX_PHASE_EWALD, s);
        RSX_CK(rsx::launch_ewald<float>(pk, g.nx, g.ny, g.nz, (const Geo<float>*)c->geo, c->twz,
                                        true, dc, c->img, s, c->err, c->wait_polls),
               "Ewald kernel");
      }
      PhaseTimer pt(c, RSX_PHASE_ROTATE, s);
      RSX_CK(rsx::launch_rotate_acc<float>(c->img, c->acc, g.nx, g.ny, alpha[k], rotation != 0, s),
             "rotation kernel");
    }
  }
  return RSX_OK;
}

// All angles of one energy on the z-first path (plan from zfirst_plan):
// per batch of up to kz angles, the polarisation + z-FFT pass keeps the ns
// q_z planes of every angle (packed: angle k, field f, plane s at
// ((k * 3 + f) * ns + s) * nx * ny), one launch x-transforms all their rows,
// then per angle the fused y-FFT pass picks each pixel's two bins from the
// planes, the image and the rotation follow as on the other paths.
int run_energy_zfirst(rsx_context* c, int ie, double start, double inc, int nang, int rotation,
                      const ZPlan& zp, cudaStream_t s) {
  const rsx_config& g = c->cfg;
  int rc = ensure_geo<float>(c, ie, s);
  if (rc) return rc;
  CUtensorMap tm_m;
  if (!make_tmap_m(c, &tm_m)) return fail(RSX_ERR_CUDA, "morphology tensor map");
  const PolParams<float> pp = make_params<float>(c, ie, 0.0, 0);
  const double ref = -(double)(g.n_components - 1) / (4.0 * kPi) * (double)c->N;
  const long long fstride = (long long)zp.ns * c->npix, kstride = 3 * fstride;
  const void* twx = g.nx == 1024 ? c->tw4 : g.nx == 2048 ? c->tw2k : c->twx;
  const unsigned box = g.ny == 512 ? 32 : g.ny == 2048 ? 8 : 16;
  const rsx::YzSel sel = {zp.kb, g.nz};
  // the angles spread evenly over the fewest passes of at most kz
  const int npass = (nang + zp.kz - 1) / zp.kz, per = (nang + npass - 1) / npass;
  for (int a0 = 0; a0 < nang; a0 += per) {
    const int nk = nang - a0 < per ? nang - a0 : per;
    rsx::XAngles ang;
    memset(&ang, 0, sizeof(ang));
    ang.n = nk;
    double alpha[rsx::kMaxXAngles];
    for (int k = 0; k < nk; ++k) {
      alpha[k] = rotation ? (start + inc * (a0 + k)) * (kPi / 180.0) : 0.0;
      ang.ce[k] = (float)cos(alpha[k]);
      ang.se[k] = (float)sin(alpha[k]);
    }
    {
      PhaseTimer pt(c, RSX_PHASE_POL_FFTX, s);
      RSX_CK(rsx::launch_pol_zfft_multi(&tm_m, g.nx, g.ny, g.nz, pp, ang, c->p, kstride, fstride,
                                        zp.kb, zp.ns, c->twz, c->err, c->n_sm, c->wait_polls, s),
             "polarisation + z-FFT kernel");
    }
    {
      PhaseTimer pt(c, RSX_PHASE_FFTX, s);
      RSX_CK(rsx::launch_xfft_rows(c->p, g.nx, (long long)nk * 3 * zp.ns * g.ny, twx, s),
             "x-FFT kernel");
    }
    for (int k = 0; k < nk; ++k) {
      float dc[3] = {(float)ref, 0.f, 0.f};
      if (g.frame != RSX_FRAME_LITERAL) {
        dc[0] = (float)(ref * cos(alpha[k]));
        dc[1] = (float)(ref * sin(alpha[k]));
      }
      CUtensorMap tm;
      if (!make_tmap(c, (char*)c->p + (size_t)k * kstride * sizeof(float2), 3LL * zp.ns, &tm, box,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B))
        return fail(RSX_ERR_CUDA, "q_z plane tensor map");
      long long L = 0;
      {
        PhaseTimer pt(c, RSX_PHASE_FFTY, s);
        RSX_CK(fused_yz(c, &tm, 3, &L, s, sel, zp.ns), "y-FFT + bin selection kernel");
      }
      {
        PhaseTimer pt(c, RSX_PHASE_EWALD, s);
        RSX_CK(rsx::launch_ewald_bins(c->part, g.nx, g.ny, zp.ns, L, (const Geo<float>*)c->geo,
                                      dc[0], dc[1], dc[2], (float*)c->img, s),
               "Ewald kernel");
      }
      PhaseTimer pt(c, RSX_PHASE_ROTATE, s);
      RSX_CK(rsx::launch_rotate_acc<float>(c->img, c->acc, g.nx, g.ny, alpha[k], rotation != 0, s),
             "rotation kernel");
    }
  }
  return RSX_OK;
}

template <typename R>
int run_energy_angles(rsx_context* c, int ie, double start, double inc, int nang, int rotation,
                      cudaStream_t s) {
  if constexpr (sizeof(R) == 4) {
    ZPlan zp;
    if (zfirst_plan(c, ie, &zp)) return run_energy_zfirst(c, ie, start, inc, nang, rotation, zp, s);
    if ((c->kx > 1 || c->cfg.nx == 2048) && x_multi_cap(&c->cfg) && c->n_sm > 0 &&
        ((uintptr_t)c->M & 15) == 0)
      return run_energy_angles_batched(c, ie, start, inc, nang, rotation, s);
  }
  for (int a = 0; a < nang; ++a) {
    const double alpha = rotation ? (start + inc * a) * (kPi / 180.0) : 0.0;
    int rc = scatter_angle<R>(c, ie, alpha, c->img, s);
    if (rc) return rc;
    PhaseTimer pt(c, RSX_PHASE_ROTATE, s);
    RSX_CK(rsx::launch_rotate_acc<R>(c->img, c->acc, c->cfg.nx, c->cfg.ny, alpha, rotation != 0, s),
           "rotation kernel");
  }
  return RSX_OK;
}

// All angles of one energy on the linearity path, kMaxAngleBatch at a time:
// the images of a batch in one launch, then one rotate-and-accumulate
// launch over the batch (the same sums in the same order as one launch per
// angle).
template <typename R>
int run_energy_linear(rsx_context* c, int ie, double start, double inc, int nang, int rotation,
                      cudaStream_t s) {
  const rsx_config& g = c->cfg;
  int rc = ensure_geo<R>(c, ie, s);
  if (rc) return rc;
  if ((rc = ensure_bins<R>(c, ie, s))) return rc;
  for (int a0 = 0; a0 < nang; a0 += rsx::kMaxAngleBatch) {
    rsx::AngleBatch<R> ab;
    memset(&ab, 0, sizeof(ab));
    for (int a = a0; a < nang && a < a0 + rsx::kMaxAngleBatch; ++a)
      rsx::add_angle(ab, rotation ? (start + inc * a) * (kPi / 180.0) : 0.0, g.nx, g.ny);
    {
      PhaseTimer pt(c, RSX_PHASE_EWALD, s);
      RSX_CK(rsx::launch_ewald_linear_many<R>(c->bins5, g.nx, g.ny, (const Geo<R>*)c->geo, ab,
                                              g.frame == RSX_FRAME_LITERAL, c->imgs, s),
             "Ewald kernel");
    }
    PhaseTimer pt(c, RSX_PHASE_ROTATE, s);
    RSX_CK(rsx::launch_rotate_acc_many<R>(c->imgs, c->acc, g.nx, g.ny, ab, rotation != 0, s),
           "rotation kernel");
  }
  return RSX_OK;
}

template <typename R>
int run_impl(rsx_context* c, double start, double inc, int nang, int rotation,
             const std::vector<int>& sel, void* out, int where, cudaStream_t s) {
  const size_t img_bytes = (size_t)c->npix * sizeof(R);
  // host output lands in `out` only once every energy has succeeded and no
  // pipelined kernel reported a timeout: until then it is staged in the
  // context's page-locked buffer (asynchronous downloads, no pageable copy)
  unsigned char* staged = nullptr;
  if (where == RSX_HOST) {
    const size_t need = sel.size() * img_bytes;
    if (need > c->host_stage_bytes) {
      if (c->host_stage) cudaFreeHost(c->host_stage);
      c->host_stage = nullptr;
      c->host_stage_bytes = 0;
      if (cudaHostAlloc(&c->host_stage, need, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        c->host_stage = nullptr;
        return fail(RSX_ERR_OOM, "no page-locked host memory to stage %zu result bytes", need);
      }
      c->host_stage_bytes = need;
    }
    staged = (unsigned char*)c->host_stage;
  }
  for (size_t o = 0; o < sel.size(); ++o) {
    const int ie = sel[o];
    RSX_CK(cudaMemsetAsync(c->acc, 0, img_bytes, s), "clear average");
    const int rc = c->cfg.algorithm == 3 && c->imgs
                       ? run_energy_linear<R>(c, ie, start, inc, nang, rotation, s)
                       : run_energy_angles<R>(c, ie, start, inc, nang, rotation, s);
    if (rc) return rc;
    const double inv = 1.0 / nang;  // Ewald_Avg[i] / numRotation (Algorithm 1)
    PhaseTimer pt(c, RSX_PHASE_OTHER, s);
    if (where == RSX_DEVICE) {
      RSX_CK(rsx::launch_scale<R>(c->acc, (char*)out + o * img_bytes, c->npix, inv, s),
             "average kernel");
    } else {
      RSX_CK(rsx::launch_scale<R>(c->acc, c->acc, c->npix, inv, s), "average kernel");
      RSX_CK(cudaMemcpyAsync(staged + o * img_bytes, c->acc, img_bytes, cudaMemcpyDeviceToHost, s),
             "result download");
    }
  }
  if (where == RSX_HOST) {
    RSX_CK(cudaStreamSynchronize(s), "result download");
    const int rc = take_kernel_error(c);
    if (rc) return rc;
    memcpy(out, staged, sel.size() * img_bytes);
  }
  return RSX_OK;
}
}  // namespace

int rsx_nt(rsx_context* c, int ie, void* nt_out, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_energy(c, ie))) return rc;
  if (!nt_out) return fail(RSX_ERR_INVALID, "nt_out is NULL");
  if (c->cfg.algorithm < 2)
    return fail(RSX_ERR_STATE, "N_t needs a context made with algorithm 2 or 3");
  RSX_DEVPTR(nt_out, c->dev, "nt_out");
  DeviceGuard dg(c->dev);
  cudaStream_t s = (cudaStream_t)stream;
  const double ref = -(double)(c->cfg.n_components - 1) / (4.0 * kPi);
  if (c->cfg.precision == 32) {
    if ((rc = ensure_nt<float>(c, ie, s))) return rc;
    RSX_CK(rsx::launch_nt_restore<float>(c->nt, nt_out, c->N, ref, s), "N_t output");
  } else {
    if ((rc = ensure_nt<double>(c, ie, s))) return rc;
    RSX_CK(rsx::launch_nt_restore<double>(c->nt, nt_out, c->N, ref, s), "N_t output");
  }
  return RSX_OK;
}

int rsx_check(rsx_context* c, void* stream) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  DeviceGuard dg(c->dev);
  if (!dg.ok) return fail(RSX_ERR_CUDA, "cannot select the context's device");
  RSX_CK(cudaStreamSynchronize((cudaStream_t)stream), "stream");
  return take_kernel_error(c);
}

int rsx_set_timing(rsx_context* c, int enable) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  c->timing = enable != 0;
  return RSX_OK;
}

int rsx_set_wait_limit(rsx_context* c, long long polls) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  c->wait_polls = polls < 0 ? rsx::kWaitPolls
                            : polls > 0xffffffffLL ? 0xffffffffu : (unsigned)polls;
  return RSX_OK;
}

int rsx_phase_times(rsx_context* c, double* ms, long long* launches) {
  if (!c) return fail(RSX_ERR_INVALID, "context is NULL");
  DeviceGuard dg(c->dev);
  double t[RSX_N_PHASES] = {0};
  long long n[RSX_N_PHASES] = {0};
  cudaError_t err = cudaSuccess;
  for (auto& r : c->recs) {
    float x = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, r.a, r.b);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    t[r.phase] += x;
    n[r.phase] += 1;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  if (err != cudaSuccess) return cuda_fail(err, "phase timers");
  for (int i = 0; i < RSX_N_PHASES; ++i) {
    if (ms) ms[i] = t[i];
    if (launches) launches[i] = n[i];
  }
  return RSX_OK;
}

int rsx_run(rsx_context* c, double start, double inc, double end, int rotation,
            const int* energy_idx, int n_sel, void* out, int where, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!out) return fail(RSX_ERR_INVALID, "out is NULL");
  if (where != RSX_HOST && where != RSX_DEVICE)
    return fail(RSX_ERR_INVALID, "where=%d: must be RSX_HOST or RSX_DEVICE", where);
  const int nang = rsx_angle_count(start, inc, end, rotation);
  if (nang < 1) return fail(RSX_ERR_INVALID, "angle list [%g, %g, %g] is empty or invalid", start, inc, end);
  std::vector<int> sel;
  if (energy_idx) {
    if (n_sel < 0) return fail(RSX_ERR_INVALID, "n_sel < 0");
    for (int i = 0; i < n_sel; ++i) {
      if ((rc = check_energy(c, energy_idx[i]))) return rc;
      sel.push_back(energy_idx[i]);
    }
  } else {
    for (int i = 0; i < (int)c->energies.size(); ++i) sel.push_back(i);
  }
  if (sel.empty()) return RSX_OK;
  if (where == RSX_DEVICE) RSX_DEVPTR(out, c->dev, "device output");
  DeviceGuard dg(c->dev);
  cudaStream_t s = (cudaStream_t)stream;
  return c->cfg.precision == 32 ? run_impl<float>(c, start, inc, nang, rotation, sel, out, where, s)
                                : run_impl<double>(c, start, inc, nang, rotation, sel, out, where, s);
}

