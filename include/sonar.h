/*
 * sonar.h — C ABI of the GB300 (sm_103a) per-ping coherent echo-formation library.
 *
 * The library forms the volumetric output of a 3D sonar ("Towards Realistic 3D Sonar
 * Simulation", Sec. II.A: an azimuth x elevation x range intensity volume and a point
 * cloud) by phase-aware signal formation (Sec. II.B): rays cast into a triangle mesh
 * along direct, refracted (Sec. II.A, Snell in a sound-speed profile) and mirror
 * multipath routes; per-hit backscatter with speckle; complex baseband echoes per
 * receive element with the phase set by the two-way delay; coherent summation into
 * beams. The sampling grid follows Sec. III Eq. 1-3 (cell-centred beams and bins).
 *
 * Conventions
 *  - World frame z up, sea surface at z = surface_z. Sonar frame x forward, y left,
 *    z up. A pose rotates sonar-frame vectors into the world frame.
 *  - Every function returns SONAR_OK (0) or a negative SONAR_E_* code; the message of
 *    the last failure is available from sonar_last_error().
 *  - All GPU work of a call is enqueued on the context stream. Calls that return host
 *    results (cloud counts, debug exports) synchronise that stream before returning.
 *  - Output buffers belong to the caller and may be device or host memory (pageable
 *    or pinned); host outputs are filled by a device-to-host copy inside the call.
 *    Input arrays are host memory and are copied during the call.
 *  - One context per host thread; a context is bound to one device.
 */
#ifndef SONAR_H
#define SONAR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SONAR_API __attribute__((visibility("default")))
#else
#define SONAR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- error codes */
#define SONAR_OK 0
#define SONAR_E_ARG (-1)          /* invalid argument or parameter combination */
#define SONAR_E_NOMEM (-2)        /* device or host allocation failed */
#define SONAR_E_CUDA (-3)         /* CUDA runtime or driver error */
#define SONAR_E_CAPACITY (-4)     /* caller buffer too small; needed size in last_error */
#define SONAR_E_TIMEOUT (-5)      /* a device-side bounded wait or loop hit its limit */
#define SONAR_E_NOSCENE (-6)      /* sonar_ping before sonar_scene_upload */
#define SONAR_E_UNSUPPORTED (-7)  /* parameters outside what the kernels implement */

/* ---------------------------------------------------------------- precision forms */
/* Beamforming contraction precision. Every form accumulates in FP32 on the tensor
   cores. Route geometry, delays and carrier phase carry FP64-grade precision: FP64 on
   the curved-ray and field routes, FP32 pairs (hi + lo, about 48 significant bits) on
   the straight-ray route, delays within 1e-12 relative of FP64 either way; hit
   amplitudes are FP32 and echoes are synthesised with FP32 accumulation.
   SONAR_FP32: each operand split into BF16 hi + lo, three products hi*hi + hi*lo +
               lo*hi (relative operand error ~2^-17).
   SONAR_BF16 / SONAR_FP16: one product of BF16 / FP16 operands. */
#define SONAR_FP32 0
#define SONAR_BF16 1
#define SONAR_FP16 2

/* ---------------------------------------------------------------- types */
typedef struct sonar_ctx sonar_ctx;

/* Sonar pose: position t (world, metres) and unit quaternion q = (w, x, y, z). */
typedef struct {
  double t[3];
  double q[4];
} sonar_pose;

/* Sound-speed profile c(z), z up. n_nodes = 0: isovelocity at params.c_ref;
   1: isovelocity at c[0]; 2: one linear gradient through (z[0], c[0]), (z[1], c[1]),
   extended linearly (curved rays, Sec. II.A). Host pointers. */
typedef struct {
  int32_t n_nodes;
  const double* z;
  const double* c;
} sonar_ssp;

/* Sensor and run parameters. Beams and rays are cell-centred grids over the fields
   of view (Sec. III Eq. 2-3); range bins are n_range cells of (r_max - r_min)/n_range
   (Eq. 1), sampled at their centres. */
typedef struct {
  int32_t nx, ny;            /* receive elements along sonar y and z (nx % 4 == 0) */
  double pitch_m;            /* element pitch */
  double f0_hz, bw_hz;       /* carrier and LFM bandwidth */
  double pulse_s;            /* pulse length T_p (Hann-windowed up-chirp) */
  double c_ref;              /* sound speed of range bins and steering; <= 0: c(z_sonar) */
  double hfov_rad, vfov_rad;
  int32_t n_beam_az, n_beam_el, n_range;
  double r_min_m, r_max_m, r_blank_m;
  int32_t n_ray_az, n_ray_el, n_sub;  /* rays per cell grid; n_sub in {1, 4} jittered */
  int32_t max_bounces;                /* specular reflections per route, 0..3 */
  double surface_z;                   /* NaN: no sea surface */
  double r_surface, r_seabed;         /* reflection coefficients (surface, mirror tris) */
  double alpha_np_per_m;              /* amplitude attenuation */
  uint64_t seed;                      /* speckle / jitter hash seed */
  int32_t precision;                  /* SONAR_FP32 | SONAR_BF16 | SONAR_FP16 */
  int32_t thr_mode;                   /* 0: absolute threshold, 1: relative to ping max */
  double thr;
  const float* taper;                 /* host [ny][nx] element weights; NULL = uniform */
} sonar_params;

/* One point of the cloud: strongest return of a beam (Sec. II.A point-cloud output). */
typedef struct {
  float x, y, z, intensity;
  int32_t beam, bin;
} sonar_point;

/* Debug/parity export of one hit (32 bytes). key: mesh hits ((ray * n_sub + sub) << 2
   | bounce), plus 0x40000000 for the cross term that returns straight (arriving from the
   hit) or 0x20000000 for its reciprocal (arriving along the route); point scatterers
   0x80000000 | (point << 8) | route, cross pairs 0xC0000000 | (point << 16) |
   (out route << 8) | back route (SONAR_OPT_CROSS); water-column scatterers
   0xA0000000 | index (sonar_set_volume). */
typedef struct {
  uint32_t key;
  int32_t prim;   /* triangle id, or -1 for a point scatterer */
  double tau;     /* two-way delay [s] (FP64) */
  float amp, phi; /* |c_k| and arg c_k */
  float uy, uz;   /* sonar-frame arrival direction (y, z) */
} sonar_hit;

/* Counters of the last ping or batch. */
typedef struct {
  int64_t n_hits;            /* hits over all pings */
  int64_t hit_capacity;
  int32_t n_pings;
  int32_t taps;              /* pulse-window taps per hit */
  int32_t kernels;           /* kernel launches of the last call */
  /* per-stage device time of the last call (CUDA events on the work stream, recorded
     only with SONAR_OPT_TIMING): ray casting, binning, synthesis, operand conversion,
     beamforming GEMM, peak extraction */
  float ms_trace, ms_bin, ms_synth, ms_convert, ms_beamform, ms_peaks;
  /* tiles of the last synchronous call: beamforming N tile, synthesis tile width in
     complex columns (0: the kernel's default or a kernel without tile widths), and 1
     when the autotuner chose them */
  int32_t tile_n, synth_cols, autotuned;
  /* tensor flops the z-split synthesis kernel's MMAs executed in the last synchronous
     call (2 M N K per MMA, every product of the FP32 form counted; 0 for the other
     synthesis kernels) */
  double synth_mma_flop;
  /* CTAs per cluster of the beamforming contraction in the last synchronous call (1, 2
     or 4; SONAR_OPT_GEMM_CLUSTER) */
  int32_t gemm_cluster;
  /* 1 when the last synchronous call formed separable beams (SONAR_OPT_BEAMFORM), 0 for
     the dense contraction */
  int32_t beam_sep;
} sonar_stats;

/* ---------------------------------------------------------------- context */
/* Creates a context on `device` that enqueues on `cuda_stream` (a cudaStream_t; NULL
   is the legacy default stream). Fails with SONAR_E_UNSUPPORTED on a device that is
   not sm_103. The context owns the scene, BVH, steering matrix and workspaces. */
SONAR_API int sonar_create(sonar_ctx** out, int device, void* cuda_stream);
SONAR_API int sonar_set_stream(sonar_ctx* ctx, void* cuda_stream);
/* Frees every resource of the context (after synchronising its stream). NULL is ok. */
SONAR_API int sonar_destroy(sonar_ctx* ctx);
/* Message of the last failure of this context ("" if none). Valid until the next call. */
SONAR_API const char* sonar_last_error(const sonar_ctx* ctx);

/* Options. SONAR_OPT_DEBUG: 1 keeps FP64 delays of hits and element echoes of the
   last call for sonar_get_hits / sonar_get_echoes. SONAR_OPT_TIMING: 1 records
   per-stage CUDA events on the work stream and reports the stage times in
   sonar_stats; calls then launch their kernels directly instead of replaying the
   graph (graph event nodes cannot be timed).
   SONAR_OPT_GRAPH: 1 (default) replays the ping pipeline as a captured CUDA graph.
   SONAR_OPT_TILE_N: beamforming N tile (128, 192, 224 or 256); 0 (default) picks per
   call the width that minimises waves x width, waves being the output tiles over the
   SMs rounded up. */
#define SONAR_OPT_DEBUG 1
#define SONAR_OPT_TIMING 2
#define SONAR_OPT_GRAPH 3
#define SONAR_OPT_TILE_N 4
/* SONAR_OPT_SYNTH: 0 (default) synthesises element echoes on the tensor cores where the
   array allows it (nx a power of two, and either nx ny a multiple of 128, where the
   z phasor splits into coarse and fine factors, or ny % 8 == 0 and ny <= 32), 1 always
   uses the FP32 SIMT synthesis kernel. 2, 3 and 4 are as 0 but ask the z-split
   tensor-core kernel for tiles of 32, 64 or 96 complex columns; a shape that does not
   fit the array and pulse falls back to the default choice. Any other value:
   SONAR_E_ARG. */
#define SONAR_OPT_SYNTH 5
/* SONAR_OPT_RAW: 0 (default) synthesises the element echoes already pulse-compressed,
   through the pulse autocorrelation R (Sec. II.B). U = 1..8 instead synthesises the raw
   element time series, the echo of the transmitted chirp p itself, at U samples per
   range cell (t_n + s dt / U, s < U: a sampling rate of U / dt >= B), and compresses it
   with an explicit matched filter (correlation with p) before beamforming. The result
   equals the compressed echoes to the quadrature error of the correlation sum (about
   2e-4 relative at U = 4, 4e-5 at U = 6). Costs U synthesis passes. Needs a pulse longer
   than two range samples (SONAR_E_UNSUPPORTED otherwise); any other value: SONAR_E_ARG. */
#define SONAR_OPT_RAW 6
/* SONAR_OPT_BVH: how sonar_scene_upload builds the triangle hierarchy. 0 (default): a
   top-down binned surface-area-heuristic build on the host (fewer node visits per ray;
   sequential host work, once per scene); 1: Morton-order LBVH built on the device (the
   fastest build). Both give the same hits; takes effect at the next upload. */
#define SONAR_OPT_BVH 7
/* SONAR_OPT_CROSS: 1 adds out/back cross-term multipath (Sec. II.B multi-bounce and
   secondary paths, with the outgoing and returning legs allowed to differ); 0 (default)
   keeps every route monostatic (the same legs out and back).
   Mesh: every hit reached after k >= 1 reflections adds two echoes, out along the route
   and straight back to the array and the reciprocal, when the straight leg reaches the
   facet from the side the route arrives on and passes no other triangle closer than
   0.1 mm to the hit. Delay (L + L_d) / c for route length L and straight distance L_d;
   amplitude Gamma sqrt(mu cos(k_d) dOmega) / L_d exp(-alpha (L + L_d)) (bistatic
   Lambertian scattering over the route's footprint, Gamma the route's one-way
   reflection product, k_d the straight leg's incidence angle); one speckle phase for the
   pair. Point scatterers: every ordered pair (i, j) of distinct valid image-source
   routes adds out along i and back along j, delay (L_i + L_j) / c, amplitude
   sigma Gamma_i Gamma_j / (L_i L_j) exp(-alpha (L_i + L_j)), arriving along j.
   Isovelocity profiles only (SONAR_E_UNSUPPORTED at the ping with a gradient);
   at most 2^27 sub-rays and 16384 point scatterers. Any other value: SONAR_E_ARG. */
#define SONAR_OPT_CROSS 8
/* SONAR_OPT_AUTOTUNE: 1 (default) lets the first synchronous call of each shape (ping
   count, range and beam grids, array, precision, raw phases, pulse and range extent) time
   the beamforming N tiles 256, 224, 192 and 128 and, for arrays the z-split synthesis
   serves, its tile widths 96, 64 and 32 complex columns on this device (per-stage events,
   the best of three runs of the call's own pings), and keeps the fastest of each for
   every later call of that shape (an asynchronous call of a new shape first makes one
   synchronous call). Only choices left to the library are tuned: SONAR_OPT_TILE_N and
   SONAR_OPT_SYNTH, when set, win. 0: the closed-form tile heuristic. */
#define SONAR_OPT_AUTOTUNE 9
/* SONAR_OPT_TRAVERSAL: how straight rays (isovelocity, no cross terms) traverse the
   hierarchy. 0 (default): one sub-ray per thread, each with its own stack. 1:
   warp-cooperative: the 32 sub-rays of a warp walk one shared stack in lockstep, a node
   visited when any lane's ray overlaps it. Both give the same hits. Any other value:
   SONAR_E_ARG. */
#define SONAR_OPT_TRAVERSAL 10
/* SONAR_OPT_TTD: 0 (default) forms phase-shift beams (Sec. II.B coherent summation:
   one phase per element and beam). U = 1..8 forms true-time-delay beams instead, for
   wide apertures in range- and depth-dependent settings (Sec. II.A): the element echoes
   are synthesised wideband, with the plane-wave delay u_k . p_m / c of each hit across
   the aperture kept in the envelope as well as in the carrier phase,
     s_m(t) = sum_k c_k exp(j k_a u_k . p_m) R(t - tau_k + u_k . p_m / c),
   at U phases t_n + s dt / U per range cell, and each beam reads every element at its
   own steering delay -u_b . p_m / c by 4-point Lagrange interpolation on that grid:
     B_b(t_n) = sum_m W_bm sum_q h(x_bm - q) s_m(t_n + q dt / U),
   x_bm = -U u_b . p_m / (c dt), h the Lagrange kernel and W_bm the phase-shift weights.
   The interpolation error falls with the fourth power of the grid spacing (about 4e-4
   of the beam energy at U = 4 on a 20 us range grid). The levels q run as extra
   column blocks of the steering operand, so the beamformer stays one tensor-core
   contraction, its K dimension (levels) times longer; sonar_get_raw returns the
   wideband phases and sonar_get_echoes phase 0. FP32 and BF16 forms only, at most 64 x
   64 elements, not with SONAR_OPT_RAW (SONAR_E_UNSUPPORTED at the ping); any other
   value: SONAR_E_ARG. */
#define SONAR_OPT_TTD 11
/* SONAR_OPT_GEMM_CLUSTER: how many CTAs share each steering tile of the beamforming
   contraction by multicast. 0 (default) chooses, as measured fastest: for the FP32
   form 2 where two divide the row tiles (128 range samples each, over all pings of the
   call), else 1; for the BF16 and FP16 forms 1; for the second stage of separable beams
   (SONAR_OPT_BEAMFORM, one K block per tile) 1. 1, 2 or 4 ask for that size, which falls
   back to 1 where it does not divide the row tiles (4 moves the least operand data but
   measured slower than 2: every stage waits for the slowest of the four CTAs). The results agree to the rounding
   of the element echoes (the synthesis adds with atomics in any order). Any other value:
   SONAR_E_ARG. */
#define SONAR_OPT_GEMM_CLUSTER 12
/* SONAR_OPT_BEAMFORM: 0 (default) forms phase-shift beams in two stages where the
   steering matrix factors (Sec. II.B coherent summation, the same sum regrouped): with a
   separable taper w_m = wy[my] wx[mx] the steering phase splits into a row part that
   depends only on the beam's elevation (u_z = sin el) and a column part, so
   B[el, az](t) = sum_mx wx e^{-j k_a u_y y_mx} U[el](t, mx) / sum w, with
   U[el](t, mx) = sum_my wy e^{-j k_a u_z z_my} s_(my, mx)(t): a contraction over the
   array's rows per elevation (FP32 on the CUDA cores) and one over its columns per beam
   (the tensor-core GEMM with K = 2 nx), nx (1 + ny / n_beam_az) complex multiply-adds
   per beam and range sample instead of nx ny (C2: 40 against 1024). It applies to
   phase-shift beams (not SONAR_OPT_TTD), a separable taper (NULL, or one that a product
   of a row and a column reproduces to 1e-6 of its largest weight), the FP32 and BF16
   forms, arrays of at most 32 columns and 64 rows with an even element count and
   n_beam_el ny <= 4096, and beam grids whose rows hold a multiple of 64 beams (the
   GEMM's N tile, 256 or 128, then lies in one elevation row; the caller's
   SONAR_OPT_TILE_N wins). Elsewhere the dense contraction runs. 1: always the dense
   contraction. sonar_get_stats reports which one the last call used. */
#define SONAR_OPT_BEAMFORM 13
SONAR_API int sonar_set_option(sonar_ctx* ctx, int32_t option, int64_t value);

/* ---------------------------------------------------------------- scene */
/* Uploads a static scene (Sec. II.A ray casting target) and builds its BVH: by
   default a binned-SAH hierarchy built on the host and refitted and packed on the
   device; with SONAR_OPT_BVH 1 a Morton-order LBVH built entirely on the device.
   verts [n_verts][3] f32 (metres); tris [n_tris][3] i32 vertex indices; mu [n_tris]
   backscatter coefficient; flags [n_tris] bit0 = specular mirror
   (reflects with r_seabed); points [n_points][3] f32 point scatterers with amplitude
   coefficients sigma [n_points]; planes [n_planes][4] f64 unit normal and offset
   (n.x = d) of mirror planes used for point-scatterer image routes. Any count may be
   0 (its pointers may then be NULL). Replaces a previous scene. */
SONAR_API int sonar_scene_upload(sonar_ctx* ctx, const float* verts, int64_t n_verts, const int32_t* tris,
                       int64_t n_tris, const float* mu, const uint8_t* flags, const float* points,
                       const float* sigma, int64_t n_points, const double* planes, int64_t n_planes);

/* Water-column (volume) reverberation (Sec. II.B volumetric backscatter paths): n point
   scatterers frozen in the world frame, uniform in the box [lo, hi]. Scatterer i sits at
   lo + (hi - lo) u, u the first three 24-bit fractions (word >> 8) / 2^24 of the 32-bit
   pcg4d hash (Jarzynski & Olano 2020) of (i mod 2^32, i div 2^32, 0x564F4C,
   seed ^ seed >> 32), seed the ping's params.seed. Each has the amplitude coefficient
   sigma = sqrt(s_v V / n), V the box volume, so that the backscattering cross-section per
   unit volume is s_v [1/m]; it echoes on its direct route when the straight leg to the
   array is clear: amplitude sigma / L^2 exp(-2 alpha L), delay 2 L / c, no speckle phase
   (the random positions make the reverberation speckle). Hit keys 0xA0000000 | i. */
typedef struct {
  int64_t n;          /* scatterers; 0 turns volume reverberation off; at most 2^28 */
  double lo[3], hi[3];/* world-frame box [m], hi > lo on every axis */
  double s_v;         /* volume backscattering coefficient [1/m], >= 0 */
} sonar_volume;
/* Sets the volume scatterers of the following pings (v NULL: none). SONAR_E_ARG for an
   empty box, a negative s_v or n outside [0, 2^28]; a ping with a sound-speed gradient,
   or with more than 2^21 point scatterers, returns SONAR_E_UNSUPPORTED while n > 0. */
SONAR_API int sonar_set_volume(sonar_ctx* ctx, const sonar_volume* v);

/* Range-dependent sound speed (Sec. II.A: rays bent by Snell's law through a range- and
   depth-dependent sound speed). c(x, z) on a regular grid of world x (range) and z
   (depth), bilinear in each cell; positions outside the grid are clamped to it (c
   constant outward). Rays are integrated by classical Runge-Kutta steps of step_m in
   arc length on (r, t, T): dr/ds = t, dt/ds = ((grad c . t) t - grad c) / c,
   dT/ds = 1 / c, the tangent renormalised after each step; the chord of each step is
   intersected with the scene and the sea surface, a hit's time and arc length
   interpolated linearly along its chord, and a reflection reflects the interpolated
   tangent. While a field is set it replaces the sonar_ssp of the pings; the reference
   speed is params.c_ref, or c at the sonar when that is <= 0. Point scatterers do not
   echo in a field (no eigen-ray search), and cross terms and volume scatterers are not
   formed (SONAR_E_UNSUPPORTED at the ping). */
typedef struct {
  int32_t nx, nz;         /* grid nodes along x and z, >= 2 each; nx = 0 removes the field */
  double x0, dx, z0, dz;  /* first node and spacing [m], dx, dz > 0 */
  const double* c;        /* host [nz][nx] sound speed [m/s], > 0; copied by the call */
  double step_m;          /* integration step in arc length [m], > 0 */
} sonar_field;
/* Sets (or, with f NULL or f->nx 0, removes) the field of the following pings.
   SONAR_E_ARG for a bad grid, speed or step. */
SONAR_API int sonar_set_field(sonar_ctx* ctx, const sonar_field* f);

/* ---------------------------------------------------------------- pings */
/* One ping. env: [n_beam_el][n_beam_az][n_range] f32 envelope |B| * TVG. cloud: up to
   cloud_cap points ordered by beam (may be NULL with cloud_cap 0). Outputs may be device
   memory, pinned host memory mapped into the device's address space (cudaHostAlloc,
   cudaHostRegister: the kernels write it in place, so results reach the host while the
   pipeline runs), or other host memory (staged on the device, copied at the end). The
   call returns when the outputs are complete. n_cloud (host, may be NULL): number of
   points found, even when it exceeds cloud_cap (then SONAR_E_CAPACITY is returned and
   cloud holds the first cloud_cap points). */
SONAR_API int sonar_ping(sonar_ctx* ctx, const sonar_pose* pose, const sonar_params* params,
               const sonar_ssp* ssp, float* env, sonar_point* cloud, int64_t cloud_cap,
               int64_t* n_cloud);

/* n_pings pings along a trajectory in one pipeline (every stage runs over all pings in
   one launch; the sequence replays as one CUDA graph). env: [n_pings][n_beam_el]
   [n_beam_az][n_range]; cloud: [n_pings][cloud_cap_per_ping]; n_cloud: host
   [n_pings]. */
SONAR_API int sonar_ping_batch(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings,
                     const sonar_params* params, const sonar_ssp* ssp, float* env,
                     sonar_point* cloud, int64_t cloud_cap_per_ping, int64_t* n_cloud);

/* Asynchronous pings for a stream of poses known one step at a time: enqueues what
   sonar_ping_batch computes and returns without waiting for it. env and cloud must be
   device memory or pinned host memory (cudaHostAlloc / cudaHostRegister; other host
   memory: SONAR_E_ARG). An envelope bound for pinned host memory is written to a device
   staging buffer and copied by a copy engine, overlapping the next ping's ray casting
   and synthesis. At most two calls are in flight: a call first waits for the one made two
   calls earlier and retires it (fills its n_cloud, host [n_pings], and returns that
   call's error, if any, in place of its own SONAR_OK). The outputs of a call are complete,
   and must not be touched before, once it is retired: by the second following
   sonar_ping_async, by sonar_wait, or by any other call on the context (all of which
   retire every call in flight first). The context's cuda_stream is ordered after a
   call's outputs once the call is retired (earlier, it would chain the next call's work
   behind this call's copy). */
SONAR_API int sonar_ping_async(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings,
                     const sonar_params* params, const sonar_ssp* ssp, float* env,
                     sonar_point* cloud, int64_t cloud_cap_per_ping, int64_t* n_cloud);
/* Retires every asynchronous call in flight, oldest first; returns the first error. */
SONAR_API int sonar_wait(sonar_ctx* ctx);
/* Failure-detection check. Runs one bounded device-side wait on an mbarrier that nothing
   completes, through the same wait code the tensor-core and bulk-copy kernels use (their
   limit is 2^31 SM cycles, about a second), here with a limit of limit_cycles (1 .. 2^31;
   2^22 is about 2 ms at 2 GHz). The wait gives up at its limit, sets the context's device
   error word and returns, so the call returns SONAR_E_TIMEOUT with its message and the
   context stays usable; SONAR_OK would mean the wait ended before its limit. Retires
   calls in flight first. SONAR_E_ARG for a limit outside the range. */
SONAR_API int sonar_probe_wait_limit(sonar_ctx* ctx, int64_t limit_cycles);

/* ---------------------------------------------------------------- debug / parity */
/* Hits of the last call (requires SONAR_OPT_DEBUG). host_out [cap]; *n = total. */
SONAR_API int sonar_get_hits(sonar_ctx* ctx, sonar_hit* host_out, int64_t cap, int64_t* n);
/* Element echoes s_m[n] of the last call (requires SONAR_OPT_DEBUG), host
   [n_pings][n_range][ny*nx][2] f32 (m = my * nx + mx). */
SONAR_API int sonar_get_echoes(sonar_ctx* ctx, float* host_out, int64_t cap_floats);
/* Raw element series of the last call, phase s of SONAR_OPT_RAW = U (requires
   SONAR_OPT_DEBUG and a ping with U > 0): r_m(t_n + s dt / U), host
   [n_pings][n_range][ny*nx][2] f32; after a true-time-delay ping (SONAR_OPT_TTD = U)
   the wideband element echoes s_m(t_n + s dt / U) instead. SONAR_E_ARG for a phase
   outside [0, U). */
SONAR_API int sonar_get_raw(sonar_ctx* ctx, int32_t phase, float* host_out, int64_t cap_floats);
SONAR_API int sonar_get_stats(const sonar_ctx* ctx, sonar_stats* out);

/* ---------------------------------------------------------------- learned surrogate */
/* The paper proposes learned scattering functions in place of costly echo physics
   (Sec. II.B). The surrogate is a per-beam 1-D convolutional network that maps a cheap
   geometric rendering of each beam to the coherent envelope profile the plain method
   forms; the plain method generates its training data, judges its error
   (sonar_sur_compare) and remains the fallback (the surrogate covers isovelocity
   scenes only and returns SONAR_E_UNSUPPORTED otherwise).
   Rendering: one ray per beam along the beam centre, routed by the plain method's
   straight-ray rules (mirror facets and the sea surface reflect, at most max_bounces);
   per beam the first two scatter (triangle) hits as (L, kappa, mu, Gamma): one-way
   route length [m], incidence cosine, facet reflectivity, one-way reflection product;
   zeros where absent.
   Network: a hit at one-way length L is splatted linearly onto range bins at bin
   coordinate (L - r_min) / dr - 1/2; four input channels (first-hit splat, second-hit
   splat, incidence cosines, reflectivities); six convolutions along range, kernel 9,
   zero padding at the beam's ends, channels 4 -> 64 -> 64 -> 64 -> 64 -> 64 -> 1, ReLU
   after the first five; output E / e_scale. BF16 weights (rounded from FP32 master
   parameters), FP32 accumulation, BF16 activations between layers, FP32 biases.
   Parameters: one FP32 vector of SONAR_SUR_N_PARAMS, layer by layer W_l [cout][cin][9]
   then b_l [cout].
   Training: mean squared error between the output and E_target / e_scale over every
   (beam, bin) of the selected beams, Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias
   correction). Needs n_range a multiple of 256. */
#define SONAR_SUR_N_PARAMS 150657

/* Sets the network parameters (host [n], n = SONAR_SUR_N_PARAMS, finite) and the output
   scale e_scale > 0; resets the Adam moments and step count. */
SONAR_API int sonar_sur_set_weights(sonar_ctx* ctx, const float* params, int64_t n, double e_scale);
/* Copies the current parameters to host [n]. SONAR_E_ARG before any set_weights. */
SONAR_API int sonar_sur_get_weights(sonar_ctx* ctx, float* params, int64_t n);
/* Geometric rendering of n_pings poses: feat [n_pings][n_beam_el * n_beam_az][8]
   (L1, kappa1, mu1, Gamma1, L2, kappa2, mu2, Gamma2), device or host memory. Needs a
   scene; SONAR_E_UNSUPPORTED for a sound-speed gradient or field. */
SONAR_API int sonar_sur_render(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings, const sonar_params* params,
                               const sonar_ssp* ssp, float* feat);
/* The surrogate's envelope of n_pings poses: env [n_pings][n_beam_el][n_beam_az][n_range]
   f32, e_scale times the network output (device memory, or host memory staged through
   the device). Returns when env is complete. */
SONAR_API int sonar_sur_ping(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings, const sonar_params* params,
                             const sonar_ssp* ssp, float* env);
/* The rendering turned into an envelope without the network (the geometric form the
   surrogate starts from, a cheap LiDAR-like sonar): env [n_pings][n_beam_el][n_beam_az]
   [n_range] f32, E[n] = TVG(r_n) sum_h a_h |R(t_n - 2 L_h / c_ref)| over the beam's two
   rendered hits, a_h = Gamma_h^2 sqrt(mu_h kappa_h dOmega_b) / L_h exp(-2 alpha L_h)
   (the plain method's Lambertian amplitude of a ray tube of the beam cell's solid angle
   dOmega_b), R the pulse autocorrelation. Device or host memory. Needs no weights. */
SONAR_API int sonar_sur_geometric(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings,
                                  const sonar_params* params, const sonar_ssp* ssp, float* env);
/* One training step on n_pings poses whose plain envelopes are env_target (device
   [n_pings][n_beam_el][n_beam_az][n_range], e.g. from sonar_ping_batch): renders the
   poses, runs the network over the n_sel selected beams (beams: device int32 indices
   into the n_pings * nb rendered beams; NULL selects all of them and ignores n_sel),
   back-propagates the mean squared error and, when update != 0, takes one Adam step of
   learning rate lr. loss (host, may be NULL): the batch's mean squared error before the
   step; grad (host [SONAR_SUR_N_PARAMS], may be NULL): its gradient. SONAR_E_ARG for an
   index outside [0, n_pings * nb) (detected on the device; the step then runs with that
   beam's input and target taken as zero) or host target/index buffers. */
SONAR_API int sonar_sur_train_step(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings,
                                   const sonar_params* params, const sonar_ssp* ssp, const float* env_target,
                                   const int32_t* beams, int64_t n_sel, double lr, int32_t update, double* loss,
                                   float* grad);
/* Error of an envelope volume against the plain method's (Sec. II.B: the plain method is
   the judge of the surrogate). */
typedef struct {
  double nl2;            /* ||E - E_ref|| / ||E_ref|| over all pings */
  int64_t lit_beams;     /* beams whose reference peak reaches rel_thr of its ping maximum */
  double peak_bin_mean;  /* mean |peak bin - reference peak bin| over lit beams (bins >= r_blank) */
  double peak_within_1;  /* fraction of lit beams whose peak bin is within 1 bin */
  double peak_within_4;  /* ... within 4 bins */
  int64_t cells;         /* (beam, bin) cells whose reference reaches rel_thr of its ping maximum */
  double si, si_ref;     /* scintillation index var(I) / mean(I)^2 of I = E^2 over those cells */
} sonar_sur_metrics;
/* env, env_ref: device [n_pings][n_beam_el * n_beam_az][n_range]; the beam and range grid
   and r_blank come from params. */
SONAR_API int sonar_sur_compare(sonar_ctx* ctx, const float* env, const float* env_ref, int32_t n_pings,
                                const sonar_params* params, double rel_thr, sonar_sur_metrics* out);

/* ---------------------------------------------------------------- allocation-free cloud */
/* Point cloud of n_pings envelope volumes that are already on the device, computed
   without allocating anything. The paper has no counterpart: this exists for callers
   that cannot call cudaMalloc (code inside an allocator or memory-pool callback, a
   real-time loop with a frozen memory budget, a process that must not grow device
   memory after start-up). It needs no context.
   env: device [n_pings][n_beam_el][n_beam_az][n_range] f32 (as written by sonar_ping /
   sonar_ping_batch); params: the beam grid, range, r_blank and threshold fields are
   used; poses: host [n_pings]; cloud: device [n_pings][cloud_cap]; n_cloud: host
   [n_pings] (may be NULL), the number of points found per ping; cuda_stream: the
   stream to enqueue on (NULL = legacy default stream). The call synchronises that
   stream before returning. Gives the points of the sonar_ping call that wrote env, in
   the same beam order, with the same beams, bins and intensities; positions are formed
   in FP64 here and in FP32 by sonar_ping, so they agree to FP32 rounding.
   Scratch (per-beam peak keys, per-ping maxima and counts) lives in one file-scope
   device array of about 4 MiB that every GPU loading the library holds until the
   process exits; the call makes no cudaMalloc/cudaFree or allocating library call.
   Limits: n_pings <= 64 and n_pings * n_beam_az * n_beam_el <= 524288, otherwise
   SONAR_E_CAPACITY is returned before any work. The first call on a device resolves
   the array's device address (cudaGetSymbolAddress, with that device current); make
   that first call before any stream capture. All calls share the array: calls whose
   GPU work overlaps (other streams, other threads) race and must be serialised by the
   caller. Returns SONAR_E_ARG on bad arguments, including an env or cloud that is not
   device (or managed) memory, checked before any work; SONAR_E_CAPACITY also when a
   ping has more than cloud_cap points and a cloud buffer was given (cloud then holds the
   first cloud_cap; with cloud NULL and cloud_cap 0 the call only counts, as sonar_ping
   does); SONAR_E_CUDA on a CUDA error. */
SONAR_API int sonar_cloud_noalloc(const float* env, int32_t n_pings, const sonar_params* params,
                                  const sonar_pose* poses, sonar_point* cloud, int64_t cloud_cap,
                                  int64_t* n_cloud, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SONAR_H */
