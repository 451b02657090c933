/*
 * rsx.h -- C ABI of the GB300 P-RSoXS forward model (libprsoxs_gb300.so).
 *
 * The library simulates polarized resonant soft X-ray scattering from a
 * voxel morphology: per-voxel uniaxial dielectric tensors, the induced
 * polarisation p, its 3-D FFT, the far-field scatter projected on the Ewald
 * sphere, and the average of the detector image over rotations of the
 * beam's electric field, for a list of photon energies (Sec. 3.3 and
 * Algorithm 1 of the paper; Algorithm 2 for the memory-minimising form).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: RSX_OK (0) on success, a negative RSX_ERR_* code
 *    otherwise.  rsx_last_error() then returns a message for the failing
 *    call on this host thread.  A failing call writes none of its outputs
 *    (rsx_run with device output: see there).
 *  - Real: float when the context was created with precision 32, double with
 *    precision 64 (the paper's float4 / double4 builds, Sec. 4.1).  Complex
 *    values are (re, im) pairs of Real.
 *  - Grid: N = nx * ny * nz voxels, x fastest, then y, then z.
 *  - Device pointers are CUDA device addresses on the current device, host
 *    pointers are ordinary (pageable or pinned) host memory.  The caller owns
 *    every buffer it passes; the library owns only what the context holds.
 *  - stream: a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it in order; an entry point that writes
 *    host memory synchronises the stream before it returns.
 *  - Detector images are [ny][nx] Real in fftshift order: the pixel (iy, ix)
 *    holds q = (2 pi (ix - nx/2) / (nx D), 2 pi (iy - ny/2) / (ny D)), with D
 *    the voxel edge in nm and integer division.
 *  - Supported sizes: nx and ny in [1, 4096], nz in [1, 65535],
 *    1 <= n_components <= RSX_MAX_COMPONENTS.  Any nx and ny are
 *    transformed exactly (mixed-radix passes; a prime factor p above 7 costs
 *    an O(p) pass per element); the fastest kernels serve FP32 grids with nx
 *    and ny 512 or 1024.
 */
#ifndef RSX_H
#define RSX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSX_OK 0
#define RSX_ERR_INVALID -1     /* bad argument, size, layout or value      */
#define RSX_ERR_OOM -2         /* a device allocation failed                */
#define RSX_ERR_CUDA -3        /* a CUDA call or kernel launch failed       */
#define RSX_ERR_UNSUPPORTED -4 /* valid, but not built (e.g. size/precision) */
#define RSX_ERR_STATE -5       /* morphology or optical constants not set   */

#define RSX_HOST 0
#define RSX_DEVICE 1
#define RSX_HOST_ASYNC 2 /* rsx_set_morphology only: page-locked host memory */

#define RSX_MAX_COMPONENTS 32

/* Frame in which p <- U^T p is applied (Sec. 3.3, Algorithm 1).
 * RSX_FRAME_LITERAL: U^T rotates the components of p while the grid and the
 *   unit vector r of Eq. (3Dscatter) stay in the material frame.
 * RSX_FRAME_LAB: U^T is left out (|U^T v| = |v|), which is the same as
 *   rotating r with p; the two differ at O((q/k)^2). */
#define RSX_FRAME_LITERAL 0
#define RSX_FRAME_LAB 1

typedef struct rsx_config {
  int nx, ny, nz;     /* voxel grid                                         */
  int n_components;   /* c, the number of materials (Sec. 3.1)              */
  double voxel_nm;    /* voxel edge D in nm (voxels are cubes, Sec. 3.1)    */
  int precision;      /* 32 (float) or 64 (double)                          */
  int algorithm;      /* 1: communication-minimising (Algorithm 1)          */
                      /* 2: memory-minimising via N_t (Algorithms 2 and 3)  */
                      /* 3: Algorithm 2 restated by linearity: p~(alpha) =  */
                      /*    cos a FFT(N_t x) + sin a FFT(N_t y), five FFTs  */
                      /*    per energy instead of three per angle (exact)   */
  int frame;          /* RSX_FRAME_LITERAL or RSX_FRAME_LAB                 */
  int validate;       /* nonzero: rsx_set_morphology rejects v or s outside */
                      /* [0, 1] and non-finite angles (Sec. 3.1); the sum   */
                      /* of v over components is never checked.             */
  int angle_batch;    /* Algorithm 1: e-field angles whose p is formed from  */
                      /* one read of the morphology (1..RSX_MAX_ANGLE_BATCH; */
                      /* 0 = the largest batch whose p buffers fit in 32    */
                      /* GiB).  Each extra angle holds another 3 N complex  */
                      /* p buffer.  Used by FP32 Algorithm 1 with nx = 512   */
                      /* or 1024 (up to 8) and nx = 2048 (up to 3; larger    */
                      /* values are lowered to that); elsewhere 1.  Each     */
                      /* angle's arithmetic is unchanged (Algorithm 1's      */
                      /* angle loop, the morphology sums shared).            */
} rsx_config;

#define RSX_MAX_ANGLE_BATCH 8

typedef struct rsx_context rsx_context;

/* Create a context for one grid and material count.  Allocates the device
 * workspace: 3 N complex for p (times the angle batch), two nx*ny Real
 * images, per-pixel Ewald
 * geometry, FFT twiddle tables, for Algorithms 2 and 3 the stored N_t entries
 * (Table 2) and, for FP32 grids with ny = 512, 1024 or 2048, nx a power of
 * two of at least 16 and nz a power of two up to 1024 (at least 4 for
 * ny = 2048), the two q_z bins per
 * pixel of the fused y-FFT + z pass (up to 4 partial slots of 3 x 2 x 16
 * bytes per pixel; 5 x 2 x 16 for Algorithm 3).  *out
 * receives the handle.  Errors: RSX_ERR_INVALID (sizes, precision,
 * algorithm), RSX_ERR_OOM. */
int rsx_create(const rsx_config* cfg, rsx_context** out);

/* Free the context and all device memory it owns.  NULL is a no-op.  The
 * caller must make sure no work of this context is still running. */
int rsx_destroy(rsx_context* ctx);

/* Message for the last failing call on this host thread ("" if none).  The
 * string stays valid until the next rsx_* call on this thread. */
const char* rsx_last_error(void);

/* Device bytes rsx_create would allocate for cfg, morphology copy included
 * (Tables 1 and 2, plus the buffers listed under rsx_create).  Returns 0 for
 * an invalid cfg. */
size_t rsx_workspace_bytes(const rsx_config* cfg);

/* The angle batch in effect for ctx (rsx_config.angle_batch after the
 * default and the shape rules above), or -1 for a NULL context. */
int rsx_angle_batch(const rsx_context* ctx);

/* The z-first path of Algorithm 1 (FP32, nz = 32, 64 or 128, nx and ny =
 * 512, 1024 or 2048).  The 3-D FFT of Algorithm 1 is separable, so its z
 * transform may come first; a detector pixel reads only the two q_z bins
 * b0 = floor(q_z / dq_z) and b0 + 1 of Eq. (Ewald), and since q_z <= 0 on
 * the sphere all pixels of one energy read one cyclic run of bins ending at
 * bin 1.  On this path rsx_run forms p, transforms each pixel's z column,
 * keeps only that run's planes, and x- and y-transforms those planes
 * instead of all nz slices (the same transform values; only the rounding
 * order differs).  It serves an energy when the run holds at most 3/4 of the
 * nz bins; the angles of one morphology read are then up to
 * min(32, angle_batch * nz / n_planes), spread evenly over the passes.
 * For energy_index: *n_planes receives the run length (0 when the path does
 * not serve this context or energy), *first_bin its first bin (the run is
 * first_bin, ..., first_bin + n_planes - 1 mod nz), *angles_per_pass the
 * angles per morphology read; any of them may be NULL.  Errors:
 * RSX_ERR_INVALID (NULL context, index out of range), RSX_ERR_STATE (no
 * optical constants yet). */
int rsx_zfirst_plan(const rsx_context* ctx, int energy_index, int* n_planes, int* first_bin,
                    int* angles_per_pass);

/* The same plan (the q_z bins of Eq. (Ewald) that Algorithm 1's detector
 * pixels read) from a configuration and a photon energy in eV alone: the
 * run a context created from cfg would use for that energy (with the angle
 * batch cfg resolves to, see rsx_angle_batch, and a 16-byte aligned
 * morphology).  Host arithmetic only: needs no GPU and allocates nothing.
 * Outputs as for rsx_zfirst_plan (all 0 where the path does not serve cfg
 * or the energy).  Errors: RSX_ERR_INVALID (cfg as for rsx_create, energy
 * not finite or <= 0). */
int rsx_zfirst_plan_for(const rsx_config* cfg, double energy_ev, int* n_planes, int* first_bin,
                        int* angles_per_pass);

/* Number of e-field angles in the inclusive list start:increment:end
 * (degrees, Algorithm 1 "E_Angle [start, increment, end]"); 1 when rotation
 * is 0.  Returns -1 for increment <= 0, end < start or non-finite input. */
int rsx_angle_count(double start_deg, double increment_deg, double end_deg, int rotation);

/* Morphology M (Sec. 4.1, Fig. 3): [c][nz][ny][nx] entries of 4 Real
 * (v_frac, s, phi, theta), component-major; phi and theta in radians.
 * where = RSX_HOST: Algorithm 1 copies it into the context once.  Algorithms
 *   2 and 3 borrow it and stream one component at a time to the GPU for each
 *   energy (Algorithm 3 of the paper), so it must stay valid until the last
 *   run; pinned memory lets the copies overlap the N_t kernel.
 * where = RSX_DEVICE: borrowed, not copied; the pointer must stay valid and
 *   unchanged until the last run that uses it has finished, and must be
 *   aligned to 4 * sizeof(Real).
 * where = RSX_HOST_ASYNC (Algorithm 1): like RSX_HOST, but M must be
 *   page-locked host memory and the copy is only enqueued on `stream`: the
 *   call returns before it lands, M must stay valid and unchanged until the
 *   stream reaches that point, and runs of this context must be ordered after
 *   it (the same stream, or an event).  With one context per stream a
 *   caller can upload the next morphology while another context computes.
 *   Memory that is not page-locked returns RSX_ERR_INVALID.  Algorithms 2
 *   and 3 treat it as RSX_HOST (borrowed).
 * With validate set, a value outside the ranges of Sec. 3.1 returns
 * RSX_ERR_INVALID and leaves the previous morphology in place.
 * FP64 Algorithm 1 contexts also evaluate every voxel's director (Eq.
 * (rotBCD)) here, once, into a [c][3][N] double buffer the context holds, so
 * the runs need no sine or cosine; for RSX_DEVICE the call then waits for
 * that kernel (on `stream`), for RSX_HOST_ASYNC it is enqueued after the
 * copy. */
int rsx_set_morphology(rsx_context* ctx, const void* M, int where, void* stream);

/* Optical constants (Sec. 3.2): energies_ev[n_energies] (> 0) and
 * constants[n_energies][c][4] = (delta_par, beta_par, delta_perp, beta_perp),
 * host memory, double.  n = 1 - delta + i beta along and across the
 * extraordinary axis.  Copied. */
int rsx_set_optical_constants(rsx_context* ctx, int n_energies, const double* energies_ev,
                              const double* constants);

/* The simulation (Algorithm 1, or Algorithm 2 when the context was made
 * with algorithm 2): for each selected energy, the detector image averaged
 * over the e-field angles start:increment:end (degrees; a single angle 0
 * and no image rotation when rotation is 0).
 * energy_idx[n_sel] selects energies by index (NULL: all, in order; this is
 * the sharding hook: disjoint subsets give the matching rows bit for bit).
 * out: [n_sel][ny][nx] Real, in host or device memory per `where`.
 * Host output is staged and copied into `out` only after the stream has
 * finished every energy and no pipelined kernel reported a timeout, so a
 * failing call leaves it untouched.  Device output is written in stream
 * order, energy by energy, and the call returns before the GPU is done: a
 * launch that fails part-way leaves the rows of the energies already
 * finished written, and a pipeline timeout (rsx_set_wait_limit) is reported
 * by the next rsx_check, or by the next call with host output. */
int rsx_run(rsx_context* ctx, double start_deg, double increment_deg, double end_deg,
            int rotation, const int* energy_idx, int n_sel, void* out, int where,
            void* stream);

/* ---- per-phase device timers (the Polarization, FFT, Scatter3DEwalds and
 * Rotation timers of the breakdowns in Sec. 6) -------------------------- */
#define RSX_PHASE_POL_FFTX 0 /* polarisation fused with the x-FFT (z-first  */
                             /* path: with the z-FFT)                        */
#define RSX_PHASE_FFTY 1     /* y-FFT                                         */
#define RSX_PHASE_EWALD 2    /* pruned q_z transform + scatter + Ewald        */
#define RSX_PHASE_ROTATE 3   /* detector rotation and accumulation            */
#define RSX_PHASE_OTHER 4    /* geometry, averaging, validation, z/x FFTs     */
#define RSX_PHASE_NT 5       /* N_t of Algorithm 3 (Algorithm 2 contexts)     */
#define RSX_PHASE_FFTX 6     /* z-first path: x-FFT of the kept q_z planes    */
#define RSX_N_PHASES 7

/* enable != 0: every kernel the context launches from now on is bracketed by
 * two CUDA events on its stream (a few microseconds each); 0 stops that. */
int rsx_set_timing(rsx_context* ctx, int enable);

/* Failure-path hook (no counterpart in the paper).  The pipelined kernels
 * wait for their bulk copies on mbarriers with a bounded number of polls;
 * when a wait runs out the kernel records the fact, lets the copies it has
 * in flight land (always with the default bound), and returns, and the next
 * rsx_run with host output fails with RSX_ERR_CUDA ("a kernel pipeline wait
 * timed out").  This sets the bound of those waits for the context's later
 * launches: polls < 0 restores the default (2^22); 0 makes every such wait
 * run out at once, so the failure path can be exercised without any fault.
 * Values above 2^32 - 1 are clamped.  The context stays usable afterwards. */
int rsx_set_wait_limit(rsx_context* ctx, long long polls);

/* Completion check for the asynchronous calls (device-output rsx_run,
 * rsx_scatter_angle, the single steps): synchronises `stream`, then reads
 * and clears the context's kernel error flag.  Returns RSX_OK when no
 * pipelined kernel of this context ran out of a bounded wait since the flag
 * was last read; otherwise RSX_ERR_CUDA ("a kernel pipeline wait timed
 * out"): every device result written since then is not valid, and the
 * per-energy data the context caches (Algorithm 2's N_t, the linearity
 * path's bins, the Ewald geometry) is dropped so the next call recomputes
 * it.  The context stays usable.  (The paper runs synchronously and has no
 * counterpart.) */
int rsx_check(rsx_context* ctx, void* stream);

/* Waits for the recorded events, writes the summed device time of each
 * phase in ms to ms[RSX_N_PHASES] and the number of kernel launches to
 * launches[RSX_N_PHASES] (either may be NULL), then clears the record. */
int rsx_phase_times(rsx_context* ctx, double* ms, long long* launches);

/* ---- single steps of the path (device buffers), for checking each row -- */

/* Algorithm 3 (NrComputation, Sec. 4.3) for one energy, in a context made
 * with algorithm 2 or 3: N_t = sum_j (N_rot^j N_rot^j - I) / (4 pi), written as
 * nt_out[5][nz][ny][nx] complex = entries xx, xy, yy, xz, yz (N_t is
 * complex symmetric; zz is never used because e lies in the x-y plane).
 * A host morphology is streamed per component, as in Algorithm 3.
 * RSX_ERR_STATE for an algorithm 1 context. */
int rsx_nt(rsx_context* ctx, int energy_index, void* nt_out, void* stream);

/* Eqs. (ncorr), (nrot), (polarization) and p <- U^T p for one energy and
 * e-field angle alpha (radians): p_out [3][nz][ny][nx] complex. */
int rsx_polarization(rsx_context* ctx, int energy_index, double alpha_rad, void* p_out,
                     void* stream);

/* Forward, unnormalised 3-D DFT (sign exp(-i ...)) of each of the three
 * complex fields in p [3][nz][ny][nx], in place. */
int rsx_fft3d(rsx_context* ctx, void* p, void* stream);

/* Eqs. (3Dscatter) and (Ewald) from a full p~ [3][nz][ny][nx] complex (FFT
 * order): detector image img_out [ny][nx] Real, fftshift order, q_z
 * interpolated linearly between the two bracketing bins. */
int rsx_ewald(rsx_context* ctx, int energy_index, const void* p_tilde, void* img_out,
              void* stream);

/* Detector rotation (Sec. 4, Algorithm 1): acc[iy][ix] += img sampled at
 * U(alpha) Q with bilinear weights, zero outside the grid. */
int rsx_rotate_accumulate(rsx_context* ctx, const void* img, double alpha_rad, void* acc,
                          void* stream);

/* One pass of the hot path for one energy and angle: morphology to the
 * unrotated detector image img_out [ny][nx] Real (fftshift order), through
 * the fused polarisation + FFT kernels and the pruned q_z transform. */
int rsx_scatter_angle(rsx_context* ctx, int energy_index, double alpha_rad, void* img_out,
                      void* stream);

/* ---- allocation-free variant of rsx_scatter_angle --------------------------
 * The paper has no counterpart to this entry point.  It exists for callers
 * that cannot allocate device memory themselves (code running inside another
 * framework's memory pool, or hosts where cudaMalloc is not allowed after
 * start-up) and so cannot create a context.  It computes the same unrotated
 * detector image as rsx_scatter_angle for one energy and one e-field angle,
 * in FP32, and calls no cudaMalloc, cudaFree or allocating library routine:
 * its working memory (p, the Ewald geometry and the FFT twiddles) is one
 * fixed array of about 26 MiB inside the library, which every GPU that loads
 * the library holds until the process exits.
 *  - Limits: nx and ny powers of two <= 4096, nz <= 4096,
 *    nx*ny*nz <= RSX_NOALLOC_MAX_VOXELS and nx*ny <= RSX_NOALLOC_MAX_PIXELS;
 *    larger grids return RSX_ERR_INVALID with a message.
 *  - M: device, [c][nz][ny][nx] float4 (v, s, phi, theta), 16-byte aligned.
 *    constants: host, [c][4] double (delta_par, beta_par, delta_perp,
 *    beta_perp) at energy_ev.  img_out: device, [ny][nx] float, fftshift
 *    order.  frame: RSX_FRAME_LITERAL or RSX_FRAME_LAB.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call uses the same array and leaves its contents behind (each
 *    call rewrites everything it reads).  Calls whose GPU work overlaps (on
 *    different streams or threads) race on it: serialise them. */
#define RSX_NOALLOC_MAX_VOXELS (1 << 20)
#define RSX_NOALLOC_MAX_PIXELS (1 << 16)
int rsx_scatter_angle_noalloc(const void* M, int nx, int ny, int nz, int n_components,
                              double voxel_nm, double energy_ev, const double* constants,
                              double alpha_rad, int frame, void* img_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RSX_H */
