// Shared device-side definitions of the echo-formation library (sm_103a only).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sonar.h"

#include <utility>

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ != 1030)
#error "this library is written for sm_103a only"
#endif

namespace sonar {

constexpr int kPad = 16;          // guard rows before/after each ping's samples in S
constexpr int kRTab = 16384;      // intervals of the pulse-autocorrelation table (linear)
constexpr int kRTabS = 512;       // intervals of the small table (cubic, 2 guard entries per side)
constexpr double kEpsHit = 1e-7;  // minimum hit distance along a segment [m]
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxStack = 64;     // BVH traversal stack depth

// Device error word bits (reported as SONAR_E_TIMEOUT / SONAR_E_CAPACITY).
constexpr int kErrTimeout = 1;
constexpr int kErrStack = 2;
constexpr int kErrCapacity = 4;
constexpr int kErrLoop = 8;
constexpr int kErrIndex = 16;  // an index array named an element outside its buffer

// One hit as consumed by echo synthesis (32 bytes).
struct HitRec {
  int32_t nglob;  // ping * nr_pad + n_first + kPad: global index of the first tap's sample
  float u0;       // n_first - q: tap i samples R((u0 + i) * dt)
  float cr, ci;   // complex coefficient c_k
  float uy, uz;   // sonar-frame arrival direction
  int32_t prim;   // triangle id, -1 for points
  uint32_t key;   // route identity (see sonar_hit)
};
static_assert(sizeof(HitRec) == 32, "HitRec must be 32 bytes");

// Binary BVH node holding both children's boxes (64 bytes).
// a = (L.lo.x, L.hi.x, L.lo.y, L.hi.y), b = (R.lo.x, R.hi.x, R.lo.y, R.hi.y),
// c = (L.lo.z, L.hi.z, R.lo.z, R.hi.z), d = (left, right, -, -); a child >= 0 is an
// internal node, a child < 0 is the leaf ~child (one triangle in leaf order).
struct BvhNode {
  float4 a, b, c;
  int4 d;
};

struct DevScene {
  const float4* tri32;     // [n_tris][3]: v0, e1, e2 (leaf order), FP32 filter
  const float* triv;       // [n_tris][9]: original vertices a, b, c (leaf order), exact (pair) test
  const int32_t* tri_prim; // leaf -> original triangle id
  const float* tri_mu;     // leaf order
  const uint8_t* tri_flags;// leaf order
  const double4_32a* tri_plane;// leaf order: n = (b - a) x (c - a) in FP64 (unnormalised), n . a
  const float4* tri_plane_df;  // leaf order, [2 n_tris]: the same as FP32 pairs, hi then lo per leaf
  const float* tri_inv_n;  // leaf order: 1 / |n|
  const BvhNode* nodes;
  int32_t n_tris;
  int32_t root;            // internal node index, or ~leaf for a one-triangle scene
  const float4* points;    // x, y, z, sigma
  int32_t n_points;
  const double4_32a* planes;   // unit normal, offset
  int32_t n_planes;
};

// Per-ping pose on the device: sonar -> world rotation (row-major) and position.
struct DevPose {
  double R[9];
  double t[3];
  float t32[3];  // the position rounded to FP32, for the FP32 traversal
  float R32[9];  // the rotation rounded to FP32, for the FP32 traversal direction
  float t_lo[3]; // t - t32 and R - R32 rounded to FP32: (t32, t_lo) and (R32, R_lo) are
  float R_lo[9]; // the FP32 pairs (hi + lo) of the straight-ray path
};

static_assert(sizeof(DevPose) % 16 == 0, "poses are copied in 16-byte words");

// Everything the trace kernels need, passed by value.
// One point-scatterer image-source route, kept for cross-term pairing: one-way length L
// (0: the route is not valid), reflection product gam, sonar-frame arrival (uy, uz).
struct PtRoute {
  double L, gam;
  float uy, uz;
  int32_t len, pad;
};

struct TraceArgs {
  DevScene sc;
  const DevPose* poses;
  const double* ray_dirs;   // [n_subrays][3] sonar-frame sub-ray directions
  const float* ray_dirs32;  // the same rounded to FP32
  const float* ray_dirs_lo; // dirs - dirs32 rounded to FP32 (the FP32 pair's low part)
  const float* row_domega;  // [n_ray_el] sub-ray solid angle per elevation row
  int32_t n_pings, n_ray_az, n_ray_el, n_sub, n_subrays;
  int32_t max_bounces, has_surface, curved;
  double surface_z, r_surface, r_seabed, alpha;
  float alpha32;                 // alpha in FP32, for the amplitude
  uint32_t seed32;
  double ssp_z0, ssp_c0, ssp_g;  // c(z) = c0 + g (z - z0)
  double inv_c0;                 // 1 / c0 (isovelocity one-way time per metre)
  double two_inv_c0;             // 2 / c0 (isovelocity two-way delay per metre of path)
  double T_stop;                 // one-way time limit
  double L_stop;                 // isovelocity path-length limit T_stop c0
  float L_stop32, surface_z32;   // the same rounded to FP32, for FP32 pre-checks
  double t0, inv_dt, hw, f0;     // sample-grid mapping of delays
  double t0_dt;                  // t0 / dt
  // the same constants as FP32 pairs (hi, lo) for the straight-ray path
  float2 L_stop_df, surface_z_df, two_inv_c0_df, f0_df, inv_dt_df, t0_dt_df, hw_df;
  int32_t nr_pad;
  int32_t n_routes;              // point-scatterer routes per point
  int32_t cross;                 // 1: out/back cross-term multipath
  int32_t warp_walk;             // 1: straight rays traverse warp-cooperatively (k_trace_warp)
  PtRoute* pt_route;             // [n_pings][n_points][n_routes] with cross terms, else null
  int64_t vol_n;                 // water-column scatterers per ping (0: none)
  double vol_lo[3], vol_hi[3];   // their world-frame box
  double vol_sigma;              // amplitude coefficient of each, sqrt(s_v V / n)
  float2 vol_lo_df[3], vol_span_df[3];  // lo and hi - lo as FP32 pairs
  // range-dependent sound speed c(x, z) on a grid (fld_nx = 0: none; then `curved` selects
  // the linear profile)
  int32_t fld_nx, fld_nz;
  double fld_x0, fld_dx, fld_z0, fld_dz, fld_h;
  double fld_idx, fld_idz;       // 1 / dx, 1 / dz
  const double* fld_c;           // [fld_nz][fld_nx]
  const int32_t* vol_order;      // [vol_n] processing order (Morton order of the positions), or null
  HitRec* hits;
  int32_t* bin_counts;           // [n_pings * nr_pad] hits per first-tap row (zeroed by the caller)
  int32_t* bin_rank;             // [hit capacity] each hit's rank among its row's hits (the
                                 // histogram atomic's old count plus its place in the warp), or null
  double* dbg_tau;               // nullable: FP64 delay per hit
  unsigned long long* n_hits;    // device counter
  int64_t hit_cap;
  int* err;
};

// ------------------------------------------------------------------ small helpers
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Programmatic dependent launch: the per-ping kernels are launched so that one may start
// (its prologue: barrier set-up, tensor-memory allocation, table loads) while the
// previous one drains its last CTAs. Every such kernel calls pdl_wait() with all its
// threads before it reads anything an earlier kernel of the ping wrote; the wait returns
// once the previous kernel has completed and its writes are visible, and because every
// kernel waits before it can finish, completion is ordered along the whole chain.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// pcg4d (Jarzynski & Olano, JCGT 2020), 32-bit.
__host__ __device__ inline void pcg4d(uint32_t& x, uint32_t& y, uint32_t& z, uint32_t& w) {
  x = x * 1664525u + 1013904223u;
  y = y * 1664525u + 1013904223u;
  z = z * 1664525u + 1013904223u;
  w = w * 1664525u + 1013904223u;
  x += y * w; y += z * x; z += x * y; w += y * z;
  x ^= x >> 16; y ^= y >> 16; z ^= z >> 16; w ^= w >> 16;
  x += y * w; y += z * x; z += x * y; w += y * z;
}

__host__ __device__ inline double u24(uint32_t h) { return (double)(h >> 8) * (1.0 / 16777216.0); }

}  // namespace sonar

// Host-side launchers implemented in the .cu files.
namespace sonar {
struct BvhBuild;
// sah != 0: the hierarchy comes from a binned-SAH build on the host copies h_verts,
// h_tris; 0: Morton order and the Karras hierarchy on the device.
cudaError_t build_bvh(const float* d_verts, const int32_t* d_tris, const float* h_verts, const int32_t* h_tris,
                      int sah, const float* d_mu, const uint8_t* d_flags, int32_t n_tris, float4** tri32, float** triv,
                      int32_t** tri_prim, float** tri_mu, uint8_t** tri_flags, double4_32a** tri_plane,
                      float** tri_inv_n, BvhNode** nodes, int32_t* root, cudaStream_t st);
// dirs32 holds 6 n floats: the directions rounded to FP32, then their FP32 residuals.
cudaError_t launch_ray_table(double* dirs, float* dirs32, float* row_domega, int32_t n_ray_az, int32_t n_ray_el,
                             int32_t n_sub, double hfov, double vfov, uint32_t seed32,
                             cudaStream_t st);
cudaError_t launch_trace(const TraceArgs& a, int sm_count, cudaStream_t st);
cudaError_t launch_points(const TraceArgs& a, cudaStream_t st);
cudaError_t launch_point_pairs(const TraceArgs& a, cudaStream_t st);
cudaError_t launch_volume(const TraceArgs& a, cudaStream_t st);
// Beam-centre geometric rendering of the learned surrogate: feat [n_pings][nbe * nba][8].
cudaError_t launch_render(const TraceArgs& a, int32_t nba, int32_t nbe, double hfov, double vfov, float* feat,
                          cudaStream_t st);

struct SynthArgs {
  const HitRec* hits_sorted;
  const int32_t* sorted_n;  // first-tap row of each sorted hit (compact copy of nglob)
  const int32_t* n_valid;   // hits with at least one tap in range (binning total)
  const int32_t* bounds;    // [gridDim + 1] cost-balanced hit ranges of the z-split kernel, or null
  const float2* rtab;       // [kRTab + 1]
  float rtab_scale;         // table index per unit of (u0 + i)
  const float2* rtab_s;     // [kRTabS + 5], entry i at u = -T_p + (i - 2) 2 T_p / kRTabS
  float rtab_s_scale;
  int32_t taps;             // W
  int32_t nx, ny;
  float pitch_over_lambda;  // element pitch in carrier wavelengths (at c_ref)
  float2* S;                // [n_pings * nr_pad][M] element echoes
  int64_t total_rows;       // n_pings * nr_pad
  int32_t n_pass;           // tensor-core synthesis: 3 (BF16 hi/lo split) or 1
  int32_t cplx_taps;        // 1: rtab_s holds a complex pulse (raw series); 0: the real
                            // pulse autocorrelation (its imaginary parts are not read)
  unsigned long long* mma_flop;  // z-split kernel: tensor flops its MMAs execute (added per CTA), or null
  int* err;
};
// Counting sort of the hits by first-tap row; counts[] holds the per-row histogram (the
// trace kernels count as they emit).
// rank: each hit's rank among its row's hits (TraceArgs::bin_rank), so the records move
// without atomics.
cudaError_t launch_bin(const HitRec* hits, const unsigned long long* n_hits, int32_t n_bins, int32_t* counts,
                       int32_t* offsets, const int32_t* rank, HitRec* sorted, int32_t* sorted_n, int sm_count,
                       int32_t* bounds, int bounds_g, int row_cost, cudaStream_t st);
cudaError_t launch_synth(const SynthArgs& a, int sm_count, cudaStream_t st);
bool synth_tc_supported(int nx, int ny, int taps);
// True when the z-split tensor-core kernel (tile widths 32, 64, 96) serves the array.
bool synth_tz_applies(int nx, int ny, int taps);
cudaError_t prepare_synth_tc();
// want_pairs: complex columns per z-split tile (32, 64, 96) when that shape fits; 0 (or
// a shape that does not fit) takes the default choice.
cudaError_t launch_synth_tc(const SynthArgs& a, int want_pairs, int sm_count, cudaStream_t st);
cudaError_t launch_rtab(float2* rtab, float2* rtab_s, double pulse, double bw, cudaStream_t st);

// Wideband element echoes for true-time-delay beamforming: the plane-wave delay across
// the aperture kept in the envelope as well as in the carrier phase,
//   s_m(t) = sum_k c_k exp(j k_a u_k . p_m) R(t - tau_k + u_k . p_m / c),
// at the U phases t_n + s dt / U. R comes from a table on a grid of dt / (U F) (tab[i] =
// (R(v_i), R(v_{i+1}) - R(v_i)), v_i = v_lo + i / (U F) samples, zero outside the pulse
// support), so that every row and phase of one (hit, element) pair reads it at the same
// interpolation weight.
struct SynthWbArgs {
  const HitRec* hits_sorted;
  const int32_t* n_valid;
  const float4* tab;
  int32_t n_tab;            // entries (a multiple of 4 bytes x 4: float4)
  int32_t uf;               // table entries per range sample, U F
  int32_t f;                // table entries per phase step, F
  float tab_x0;             // table index of v = 0 minus e1 rows: (-e1 - v_lo) U F
  int32_t e1;               // window rows before a hit's first tap row
  int32_t n_phases;         // U
  int32_t nx, ny;
  float pitch_over_lambda;  // element pitch in carrier wavelengths
  float pitch_uf;           // element pitch in table entries of delay: pitch / (c dt) U F
  float2* S;                // phase s at S + s phase_stride: [n_pings * nr_pad][M]
  int64_t phase_stride;
  int64_t total_rows;
  int* err;
};
// Table of R on the fine grid: n entries, v_i = v_lo + i du (in range samples of dt).
cudaError_t launch_wtab(float4* tab, int32_t n, double v_lo, double du, double dt, double pulse, double bw,
                        cudaStream_t st);
// wt: window rows per hit (12, 16, 20 or 24).
cudaError_t launch_synth_wb(const SynthWbArgs& a, int wt, int sm_count, cudaStream_t st);
cudaError_t prepare_synth_wb();

// ------------------------------------------------------------------ learned surrogate
// Six 1-D convolutions along range (kernel 9, channels 4 -> 64 x 5 -> 1), packed into one
// FP32 parameter vector layer by layer: W_l [cout][cin][9] then b_l [cout].
constexpr int kSurC = 64;     // hidden channels
constexpr int kSurK = 9;      // kernel taps
constexpr int kSurHalo = 8;   // zero rows before and after each beam's bins in activation buffers
__host__ __device__ constexpr int sur_cin(int l) { return l == 0 ? 4 : kSurC; }
__host__ __device__ constexpr int sur_cout(int l) { return l == 5 ? 1 : kSurC; }
__host__ __device__ constexpr int64_t sur_woff(int l) {
  return l == 0 ? 0 : sur_woff(l - 1) + (int64_t)sur_cout(l - 1) * sur_cin(l - 1) * kSurK + sur_cout(l - 1);
}
__host__ __device__ constexpr int64_t sur_boff(int l) { return sur_woff(l) + (int64_t)sur_cout(l) * sur_cin(l) * kSurK; }
constexpr int64_t kSurParams = sur_woff(6);
static_assert(kSurParams == 150657, "parameter count of the surrogate network");

// Device state of the network: FP32 master parameters, Adam moments, gradients, and the
// BF16 weights in the layouts the kernels read (the first and last layers' as FP32
// values of their BF16 rounding).
struct SurNet {
  float* theta;         // [kSurParams]
  float* m;             // Adam first moment
  float* v;             // Adam second moment
  float* grad;          // [kSurParams]
  __nv_bfloat16* wf;    // hidden layers 1..4: [4][9][64 cout][64 cin], forward B operands
  __nv_bfloat16* wb;    // [4][9][64 cin][64 cout], taps reversed: backward-data B operands
  float* w_in;          // layer 0: [64][4][9]
  float* w_out;         // layer 5: [64][9]
};
// Adam step (update != 0; bias corrections bc1 = 1 - beta1^t, bc2 = 1 - beta2^t) and the
// repacking of the BF16 weight copies from the master parameters.
cudaError_t sur_pack(const SurNet& n, int update, float lr, float b1, float b2, float eps, float bc1, float bc2,
                     cudaStream_t st);
// Layer 0 from the rendering: act1 rows of the selected beams (beams: indices into the
// rendering's rows, or null for all). Sparse input: the splats of two hits per beam.
cudaError_t sur_input(const float* feat, const int32_t* beams, int64_t n_sel, int64_t n_feat, int nr, double r_min,
                      double inv_dr, const SurNet& n, __nv_bfloat16* act1, int rb, int* err, cudaStream_t st);
struct SurConvArgs {
  CUtensorMap map_x;              // input rows [n_sel * rb][64] BF16, box 64 x 136
  CUtensorMap map_w;              // B operands [9 * 64][64] BF16, box 64 x 64
  const float* bias;              // forward: [64]
  const __nv_bfloat16* mask;      // backward-data: the gradient passes where these are > 0
  __nv_bfloat16* out;
  int64_t n_tiles;
  int tiles_per_beam, rb;
  int* err;
};
// Hidden 64 -> 64 layer on the tensor cores: forward (bias, ReLU) or backward-data.
cudaError_t sur_conv(const SurConvArgs& a, bool backward, int sm_count, cudaStream_t st);
cudaError_t sur_conv_prepare();
// Output layer 5: envelope out (inference) or the loss gradient (training).
cudaError_t sur_head(const __nv_bfloat16* act5, const SurNet& n, int64_t n_sel, int nr, int rb, const float* target,
                     const int32_t* beams, int64_t n_feat, float inv_scale, float g_scale, float* g, double* loss,
                     float* env_out, float e_scale, int* err, cudaStream_t st);
cudaError_t sur_head_bwd(const __nv_bfloat16* act5, const float* g, const SurNet& n, int64_t n_sel, int nr, int rb,
                         __nv_bfloat16* dz5, cudaStream_t st);
struct SurDwArgs {
  CUtensorMap map_x;   // the layer's input rows, box 64 x 80
  CUtensorMap map_dz;  // its output gradient rows, box 64 x 80
  float* grad_w;       // [64][64][9] in the parameter packing
  float* grad_b;       // [64]
  int64_t n_kb;        // K-blocks of 64 positions: n_sel * (nr / 64 + 1)
  int kb_per_beam, nr, rb;
  int* err;
};
// Weight and bias gradients of a hidden layer on the tensor cores.
cudaError_t sur_dw(const SurDwArgs& a, int sm_count, cudaStream_t st);
// Layer-0 weight and bias gradients from the sparse input.
cudaError_t sur_l1_dw(const float* feat, const int32_t* beams, int64_t n_sel, int64_t n_feat, int nr, double r_min,
                      double inv_dr, const __nv_bfloat16* dz1, int rb, const SurNet& n, cudaStream_t st);
// Envelope of the rendering without the network: [n_beams][nr].
cudaError_t sur_geometric(const float* feat, int64_t n_beams, int nba, int nbe, double hfov, double vfov, int nr,
                          double r_min, double dr, double c_ref, double alpha, double T, const float2* rtab, int n_tab,
                          float* env, cudaStream_t st);
// Comparison of two envelope volumes [P][nb][nr]: totals[12] (doubles, zeroed by the caller).
cudaError_t sur_compare(const float* env, const float* ref, int P, int nb, int nr, int n_blank, float rel_thr,
                        unsigned* ping_max, int32_t* beam_pk, float* beam_max, double* totals, cudaStream_t st);

// Raw element series (echo before pulse compression) and its matched filter.
// launch_ptab: for each phase s < U, the transmitted pulse shifted by s dt / U, p(u + s dt
// / U), on the grids of the two synthesis tables (ptab [U][kRTab + 1], ptab_s [U][kRTabS
// + 5]), so that a synthesis pass with them writes r_m(t_n + s dt / U); and the matched
// filter's taps taps[s][D + d] = (dt / (U E)) conj(p(d dt + s dt / U)), |d| <= D.
cudaError_t launch_ptab(float2* ptab, float2* ptab_s, float2* taps, int32_t U, int32_t D, double pulse, double bw,
                        double dt, cudaStream_t st);
struct MfArgs {
  const float2* raw;        // [U] phases of [n_pings * nr_pad + guard][M], phase_stride apart
  int64_t phase_stride;
  float2* S;                // output: compressed echoes, rows kPad .. kPad + nr of each ping
  const float2* taps;       // [U][2 D + 1]
  int32_t U, D, nr, nr_pad, M, n_pings;
};
cudaError_t launch_mfilter(const MfArgs& a, cudaStream_t st);

struct ConvertArgs {
  const float2* S;          // [n_phases][n_pings][nr_pad][M], phases phase_stride elements apart
  int64_t phase_stride;
  int32_t n_pings, nr, nr_pad, nr_x, M, k_pad;
  // operand rows: per phase and ping x_rows rows, row j holding sample j - x_guard; rows
  // j < nr + 2 x_guard are written (samples -x_guard .. nr + x_guard - 1). The plain
  // path: one phase, x_rows = nr_x, x_guard = 0.
  int32_t n_phases, x_rows, x_guard;
  int32_t mode;             // SONAR_FP32 / BF16 / FP16
  float* gain;              // [n_pings] power-of-two gain applied (FP16), else 1
  void* x_hi;               // [n_phases * n_pings * x_rows][k_pad] 16-bit
  void* x_lo;               // FP32 form only
};
cudaError_t launch_convert(const ConvertArgs& a, int sm_count, cudaStream_t st);

struct SteerArgs {
  int32_t nx, ny, n_beam_az, n_beam_el, nb_pad, k_pad;
  // true-time delay: n_levels fractional-delay levels q = q0 .. q0 + n_levels - 1, each a
  // k_pad-wide block of columns weighted by lagrange4(x - q), x = -x_scale (u_y (mx - cx)
  // + u_z (my - cy)) the steering delay in units of dt / U. Phase-shift beams: n_levels
  // = 1 and ttd = 0 (weight 1).
  int32_t n_levels, q0, ttd;
  double x_scale;
  double hfov, vfov, pitch_over_lambda;
  const double2* beam_uyz;  // [n_beams] sonar-frame (u_y, u_z) of each beam centre, FP64
  const float* taper;       // device [M] or null
  double wsum, gain;
  int32_t mode;
  void* y_hi;               // [nb_pad*2][n_levels * k_pad]
  void* y_lo;
};
cudaError_t launch_steer(const SteerArgs& a, cudaStream_t st);

struct GemmArgs {
  CUtensorMap map_xh, map_xl, map_yh, map_yl;
  int32_t tiles_m, tiles_n, k_blocks, tile_n;  // k_blocks: K / 64
  // A-operand addressing. The plain path reads row tile mb at X rows mb 128 .. + 127
  // (x_kpad = K, ttd_u = 0, x_ping_rows = nr_x, x_guard = 0). True-time delay: K runs
  // over fractional-delay levels q = ttd_q0 + K / x_kpad, and level q reads phase q mod
  // ttd_u of the echoes at a row offset floor(q / ttd_u): X rows s x_phase_rows + p
  // x_ping_rows + x_guard + n + floor(q / ttd_u) for the tile's samples n of ping p.
  int32_t x_kpad, ttd_u, ttd_q0, x_ping_rows, x_guard, x_phase_rows;
  int32_t n_phase;           // products per K slice: 3 (FP32 form: hi*hi, hi*lo, lo*hi) or 1;
                             // the FP32 form's maps have 32-element K boxes, 64-byte swizzle
  int32_t f16;               // operands FP16 (1) or BF16 (0)
  int32_t nr, nr_x, n_beams, n_blank;
  float r_min, dr, alpha2;   // TVG(r) = r exp(alpha2 r)
  const float* gain;         // [n_pings]: element-echo gain (FP16 form), nullptr: 1
  float y_gain_inv;
  float* env;                // [n_pings][Nb][Nr]
  unsigned long long* peak_keys;  // [n_pings][Nb]
  unsigned int* ping_max;    // [n_pings] float bits
  // CTAs per cluster sharing each B tile by multicast: 1, 2 or 4 (map_yh / map_yl boxes
  // then hold tile_n / cluster rows), as gemm_cluster_size() gives it
  int32_t cluster;
  // Separable beams (sep_az > 0): the echo operand holds one block of x_el_rows rows per
  // beam elevation row (the echoes already summed over the array's rows for that
  // elevation), and N tile nb, whose tile_n / 2 beams lie in elevation row nb tile_n /
  // (2 sep_az), reads its rows from that block. 0: the dense contraction.
  int32_t sep_az;
  int64_t x_el_rows;
  int* err;
};
cudaError_t prepare_gemm();
// CTAs per cluster of the GEMM for this shape: for the FP32 form 2 where two divide the
// row tiles and the cluster variant fits on the device, else (and for the one-product
// forms) 1.
int gemm_cluster_size(int tiles_m, int tile_n, int n_phase, int sm_count);
// Whether clusters of cs CTAs serve this shape at all.
bool gemm_cluster_fits(int cs, int tiles_m, int tile_n, int n_phase);
cudaError_t launch_gemm(const GemmArgs& a, int sm_count, cudaStream_t st);

// First stage of the separable phase-shift beamformer. With a separable taper w_m =
// wy[my] wx[mx], the steering phase u_b . p_m = u_y y_mx + u_z z_my and u_z = sin(el)
// fixed by the beam's elevation row, B[el, az][n] = sum_mx Wx(el, az, mx) U[el][n][mx]
// with U[el][n][mx] = sum_my Fz[el][my] s_(my, mx)[n], Fz[el][my] = wy[my] exp(-j k_a
// z_my sin el). This kernel forms U (FP32 complex multiply-adds) and stores it as the
// beamforming GEMM's echo operand: row (el, ping, n) of x_el_rows = n_pings nr_x rows per
// elevation, columns (2 mx, 2 mx + 1) = (Re, Im), BF16 (plus the FP32 form's residual).
struct Sep1Args {
  const float2* S;           // [n_pings][nr_pad][M] element echoes (rows kPad + n)
  const float2* fz;          // [n_el][ny] Fz
  int32_t n_pings, nr, nr_pad, nr_x, nx, ny, n_el, k_pad;
  int32_t mode;              // SONAR_FP32 (hi + lo) or SONAR_BF16
  void* x_hi;
  void* x_lo;
  int* err;                  // error flags (a copy that never lands)
};
// Whether the first stage serves an array of nx x ny elements (nx <= 32, ny <= 64, an
// even count: the rows of S move as 16-byte pairs of elements).
bool sep1_supported(int nx, int ny);
cudaError_t launch_sep1(const Sep1Args& a, int sm_count, cudaStream_t st);

struct PeakArgs {
  const unsigned long long* peak_keys;
  const unsigned int* ping_max;
  const DevPose* poses;
  int32_t n_pings, n_beam_az, n_beam_el, nr;
  // beam and bin grid in FP32, rounded on the host: az0 = -hfov/2, daz = hfov/n_beam_az,
  // el0, del likewise, r_min and dr
  float az0, daz, el0, del, r_min, dr;
  int32_t thr_mode;
  float thr;
  sonar_point* cloud;       // [n_pings][cap]
  int64_t cap;
  long long* n_cloud;       // [n_pings]
  // the call's results for the host, written through the device mapping of pinned host
  // words (no copy after the kernel): points per ping, then hit count and error bits
  long long* n_cloud_host;
  unsigned long long* counters_host;   // [3]: hit count, error bits, synthesis tensor flops
  const unsigned long long* n_hits;    // [2]: hit count, synthesis tensor flops
  const int* err;
};
cudaError_t launch_peaks(const PeakArgs& a, cudaStream_t st);
}  // namespace sonar
