// C ABI of the echo-formation library: context, validation, workspaces, the ping
// pipeline (trace -> bin -> synthesise -> convert -> beamform -> peaks) and its
// replay as a captured CUDA graph.
#include <cudaTypedefs.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "tcgen05.cuh"

using namespace sonar;

namespace {

// One bounded wait on an mbarrier that nothing completes: the wait of the tensor-core and
// bulk-copy kernels, with the caller's limit. It gives up at the limit, flags
// kErrTimeout and returns (no fault, no hang).
__global__ void k_wait_probe(int* err, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) tc::mbar_wait_for(tc::smem_u32(&bar), 0, err, limit);
}

// Zeroes, in one launch, every buffer a call accumulates into: the element echoes S
// (16-byte stores), the per-row hit histogram, the per-beam peak keys and ping maxima,
// the hit counter and the error bits.
// Also brings the poses in: it reads the pinned pose record through its device mapping
// (pose_src, 16-byte words), so the pipeline has no copy-engine node that could queue
// behind an earlier ping's envelope copy.
__global__ void k_clear(float2* S, int64_t n_s, float2* S2, int64_t n_s2, int32_t* counts, int32_t n_bins,
                        unsigned long long* keys, int64_t n_keys, unsigned* pmax, int n_p, unsigned long long* n_hits,
                        int* err, const uint4* pose_src, uint4* pose_dst, int n_pose16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t i = t; i < n_pose16; i += stride) pose_dst[i] = pose_src[i];
  float4* S4 = reinterpret_cast<float4*>(S);  // cudaMalloc alignment
  for (int64_t i = t; i < n_s / 2; i += stride) S4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if ((n_s & 1) && t == 0) S[n_s - 1] = make_float2(0.f, 0.f);
  float4* R4 = reinterpret_cast<float4*>(S2);  // the raw series' phases (S2 may be null: n_s2 = 0)
  for (int64_t i = t; i < n_s2 / 2; i += stride) R4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if ((n_s2 & 1) && t == 0) S2[n_s2 - 1] = make_float2(0.f, 0.f);
  for (int64_t i = t; i < n_bins; i += stride) counts[i] = 0;
  for (int64_t i = t; i < n_keys; i += stride) keys[i] = 0ull;
  for (int64_t i = t; i < n_p; i += stride) pmax[i] = 0u;
  if (t == 0) {
    n_hits[0] = 0ull;  // hit count
    n_hits[1] = 0ull;  // synthesis tensor flops
    *err = 0;
  }
}

// Beamforming N tiles the GEMM is built for; 0 picks per call the one that minimises
// waves x width (waves = output tiles / SMs, rounded up): the last wave of a few large
// tiles can leave most SMs idle.
constexpr int kTiles[] = {256, 224, 192};

int pick_tile_n(int64_t nr_rows_tiles, int64_t nb, int sm_count) {
  int best = 256;
  int64_t best_cost = INT64_MAX;
  for (int bn : kTiles) {
    const int64_t nb_pad = (nb + bn / 2 - 1) / (bn / 2) * (bn / 2);
    const int64_t tiles = nr_rows_tiles * (2 * nb_pad / bn);
    const int64_t waves = (tiles + sm_count - 1) / sm_count;
    const int64_t cost = waves * bn;
    if (cost < best_cost) { best_cost = cost; best = bn; }
  }
  return best;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

struct Derived {
  double c_ref, dr, dt, t0, hw, T_stop, pitch_over_lambda, ssp_z0, ssp_c0, ssp_g, wsum, wmax;
  int taps, nr, nr_pad, nr_x, M, k_pad, nb, nb_pad, tile_n, n_phase, n_blank, n_routes, curved;
  int64_t n_subrays, hit_cap_per_ping;
  // true-time delay: fractional-delay levels q0 .. q0 + levels - 1 (steering delays in
  // units of dt / U), guard rows of the echo operand per ping, the wideband synthesis
  // window (wt rows from e1 before a hit's first tap) and its table (n_tab entries, uf
  // per range sample, f per phase, v_lo the first entry's position in samples, x0 the
  // entry of a window's first row at u0 = 0, phase 0 and no element delay)
  int ttd_q0 = 0, ttd_levels = 1, ttd_guard = 0, wb_wt = 0, wb_e1 = 0, wb_uf = 0, wb_f = 0, wb_n_tab = 0;
  double wb_v_lo = 0.0, wb_x0 = 0.0, ttd_x_scale = 0.0;
  int sep = 0;  // 1: separable beams (two stages), 0: the dense contraction
  int n_el = 0, n_az = 0;  // beam elevation rows and beams per row
};

// The taper as wy[my] wx[mx] (wx from the row of the largest weight, wy normalised to 1
// there); false when no such product reproduces it to 1e-6 of the largest weight. A
// missing taper is uniform.
bool taper_separable(const sonar_params* p, std::vector<double>* wx, std::vector<double>* wy) {
  const int nx = p->nx, ny = p->ny;
  wx->assign((size_t)nx, 1.0);
  wy->assign((size_t)ny, 1.0);
  if (!p->taper) return true;
  int m0 = 0;
  for (int m = 1; m < nx * ny; ++m)
    if (p->taper[m] > p->taper[m0]) m0 = m;
  const double t0 = p->taper[m0];
  if (!(t0 > 0)) return false;
  const int mx0 = m0 % nx, my0 = m0 / nx;
  for (int mx = 0; mx < nx; ++mx) (*wx)[(size_t)mx] = p->taper[my0 * nx + mx];
  for (int my = 0; my < ny; ++my) (*wy)[(size_t)my] = p->taper[my * nx + mx0] / t0;
  for (int my = 0; my < ny; ++my)
    for (int mx = 0; mx < nx; ++mx)
      if (fabs((double)p->taper[my * nx + mx] - (*wy)[(size_t)my] * (*wx)[(size_t)mx]) > 1e-6 * t0) return false;
  return true;
}

// One of the two in-flight slots of asynchronous pings: its own pinned pose record,
// point counts and counter words, device envelope staging and captured graph, reused
// only after the slot's previous ping has finished.
struct AsyncSlot {
  bool busy = false;
  DevPose* pose_host = nullptr;               // pinned [p_cap], mapped
  DevPose* pose_map = nullptr;
  long long* n_cloud_host = nullptr;          // pinned [p_cap], mapped
  long long* n_cloud_map = nullptr;
  unsigned long long* counters_host = nullptr;  // pinned [3]: hit count, error bits, synthesis flops; mapped
  unsigned long long* counters_map = nullptr;
  int p_cap = 0;
  float* env_stage = nullptr;
  int64_t env_cap = 0;
  cudaEvent_t ev_gemm = nullptr, ev_done = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<uint8_t> gkey;
  int graph_kernels = 0;
  // what retiring the ping hands back
  int64_t* n_cloud_user = nullptr;
  int P = 0;
  int64_t cloud_cap = 0;
  bool cloud_given = false;
};

}  // namespace

struct sonar_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;       // private work stream (capturable)
  cudaStream_t user_stream = nullptr;  // caller's stream, ordered with events
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t stage_ev[7] = {};
  int sm_count = 0;
  std::string err;
  bool debug = false, timing = false, use_graph = true;
  int tile_opt = 0;
  // autotuner: per (pings, grid, array, precision, raw phases, pulse) the beamforming N
  // tile and the synthesis tile width measured fastest on this device at the first call
  int autotune = 1;
  struct TuneEntry {
    std::vector<uint8_t> key;
    int tile_n = 0, pairs = 0;
    float ms_gemm = 0.f, ms_synth = 0.f;
  };
  std::vector<TuneEntry> tuned;
  int cur_tile_n = 0, cur_pairs = 0;  // the choice in force for the current call (0: heuristic)
  bool cur_tuned = false;
  int raw_u = 0;      // 0: compressed synthesis; U > 0: raw series at U samples per cell + matched filter
  int ttd_u = 0;      // 0: phase-shift beams; U > 0: true-time-delay beams from wideband echoes at U phases
  int last_ttd_u = 0;
  int bvh_opt = 0;    // 0: binned-SAH hierarchy (host build), 1: Morton-order LBVH (device build)
  int cross = 0;      // 1: out/back cross-term multipath
  int traversal = 0;  // straight rays: 0 one sub-ray per thread, 1 warp-cooperative
  int gemm_cluster = 0;  // beamforming CTAs per cluster: 0 automatic, else 1, 2 or 4 where it fits
  int64_t vol_n = 0;  // water-column scatterers per ping
  sonar_field fld{};  // range-dependent sound speed (fld.nx = 0: none); c points to fld_c
  double* fld_c = nullptr;  // device copy of the grid
  std::vector<double> fld_host;
  double vol_lo[3] = {0, 0, 0}, vol_hi[3] = {0, 0, 0}, vol_sigma = 0.0;
  int32_t* vol_order = nullptr;  // Morton order of the scatterers (null: index order)
  int64_t vol_order_cap = 0;
  std::vector<uint8_t> vol_key;  // (n, seed) the order was computed for
  PtRoute* pt_route = nullptr;  // point-route records for cross pairing
  int64_t ws_pt_route = 0;
  int last_raw_u = 0;
  float2* S_raw = nullptr;  // raw series: U phases of s_elems
  int64_t ws_raw = 0;
  int synth_opt = 0;  // 0: tensor-core synthesis where supported, 1: FP32 SIMT synthesis,
                      // 2, 3, 4: tensor-core synthesis asking for 32, 64, 96 columns per tile

  // scene
  bool has_scene = false;
  DevScene sc{};
  float4* tri32 = nullptr;
  float* triv = nullptr;
  int32_t* tri_prim = nullptr;
  float* tri_mu = nullptr;
  uint8_t* tri_flags = nullptr;
  double4_32a* tri_plane = nullptr;
  float* tri_inv_n = nullptr;
  BvhNode* nodes = nullptr;
  float4* points = nullptr;
  double4_32a* planes = nullptr;
  uint64_t scene_version = 0;

  // parameter-derived tables
  std::vector<uint8_t> ray_key, steer_key, rtab_key, ptab_key;
  double* ray_dirs = nullptr;
  float* ray_dirs32 = nullptr;
  float* row_domega = nullptr;
  void* y_hi = nullptr;
  void* y_lo = nullptr;
  size_t y_elems = 0;
  float2* rtab = nullptr;
  float2* ptab = nullptr;   // raw series: U shifted pulse tables (both grids), then the matched-filter taps
  float4* wtab = nullptr;   // true-time delay: the wideband synthesis table
  std::vector<uint8_t> wtab_key;
  int ptab_u = 0, ptab_d = 0;
  float* taper_dev = nullptr;
  double2* beam_uyz = nullptr;  // beam-centre direction cosines of the steering matrix
  int64_t beam_uyz_cap = 0;
  double y_gain = 1.0;
  // separable beams: Fz [n_beam_el][ny] of the first stage and the second stage's
  // steering operand (one array row, wx[mx] exp(-j k_a u_y y_mx)), keyed like the steering
  int bf_opt = 0;  // 0: separable beams where they apply, 1: always the dense contraction
  std::vector<uint8_t> sep_key;
  float2* sep_fz = nullptr;
  int64_t sep_fz_cap = 0;
  void* ysep_hi = nullptr;
  void* ysep_lo = nullptr;
  size_t ysep_elems = 0;
  float* taper_x_dev = nullptr;
  double ysep_gain = 1.0;

  // workspaces
  int p_cap = 0;
  DevPose* pose_host = nullptr;  // pinned [p]: rotation and position of each ping
  DevPose* pose_map = nullptr;   // its device mapping
  DevPose* poses = nullptr;
  HitRec* hits = nullptr;
  HitRec* sorted = nullptr;
  int32_t* sorted_n = nullptr;
  int32_t* rank = nullptr;  // each hit's rank among its row's hits, from the trace's histogram
  double* dbg_tau = nullptr;
  int64_t hit_cap = 0;
  unsigned long long* n_hits = nullptr;
  int32_t* counts = nullptr;
  int32_t* offsets = nullptr;
  int64_t keys_cap = 0;
  float2* S = nullptr;
  int64_t s_elems = 0;
  void* x_hi = nullptr;
  void* x_lo = nullptr;
  int64_t x_elems = 0;
  float* gain = nullptr;
  float* env_stage = nullptr;
  int64_t env_cap = 0;
  unsigned long long* keys = nullptr;
  unsigned int* pmax = nullptr;
  sonar_point* cloud_stage = nullptr;
  int64_t cloud_stage_cap = 0;
  long long* n_cloud_dev = nullptr;
  long long* n_cloud_host = nullptr;  // pinned
  unsigned long long* counters_host = nullptr;  // pinned: hits of the last call, error bits
  long long* n_cloud_map = nullptr;             // device mappings of the two above
  unsigned long long* counters_map = nullptr;
  int* err_dev = nullptr;
  int32_t* synth_bounds = nullptr;  // [sm_count + 1] cost-balanced synthesis hit ranges
  int64_t ws_hits = 0, ws_bins = 0, ws_s = 0, ws_x = 0;

  // captured graphs of the synchronous calls, keyed by everything they bake in (a few,
  // so that a caller alternating output buffers does not re-capture on every call)
  struct GraphEntry {
    std::vector<uint8_t> key;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    uint64_t used = 0;
  };
  std::vector<GraphEntry> graphs;
  uint64_t graph_tick = 0;

  // asynchronous pings: two slots and the copy-engine stream of their envelopes
  AsyncSlot aslot[2];
  int next_slot = 0;
  cudaStream_t copy_stream = nullptr;

  // learned surrogate
  struct Sur {
    float* params = nullptr;       // theta | m | v | grad, kSurParams each
    __nv_bfloat16* wbf = nullptr;  // forward | backward-data B operands
    float* wsmall = nullptr;       // first-layer | last-layer weights
    SurNet net{};
    bool has_weights = false;
    double e_scale = 1.0;
    int64_t step = 0;              // Adam steps taken
    float* feat = nullptr;         // rendering [P][nb][8]
    int64_t feat_cap = 0;
    DevPose* poses = nullptr;
    int64_t poses_cap = 0;
    __nv_bfloat16* buf = nullptr;  // kSurBufs activation / gradient buffers of beams_cap beams
    int64_t beams_cap = 0;
    int rb = 0;
    float* g = nullptr;            // loss gradient [n_sel][nr]
    int64_t g_cap = 0;
    double* loss = nullptr;
    double* cmp_tot = nullptr;
    unsigned* cmp_pmax = nullptr;
    int32_t* cmp_pk = nullptr;
    float* cmp_bmax = nullptr;
    int64_t cmp_cap = 0, cmp_pk_cap = 0, cmp_bmax_cap = 0;
  } sur;

  // last call
  int last_p = 0;
  Derived last_d{};
  sonar_params last_params{};
  sonar_stats stats{};
};

namespace {

int fail(sonar_ctx* c, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(sonar_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CU(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return fail(ctx, SONAR_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                           \
  } while (0)

template <typename T>
void key_add(std::vector<uint8_t>& k, const T& v) {
  const uint8_t* p = reinterpret_cast<const uint8_t*>(&v);
  k.insert(k.end(), p, p + sizeof(T));
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

int validate(sonar_ctx* ctx, const sonar_params* p, const sonar_ssp* ssp) {
  if (!p) return fail(ctx, SONAR_E_ARG, "params is NULL");
  if (p->nx < 4 || p->ny < 1 || p->nx % 4 != 0 || p->nx > 64 || p->ny > 64)
    return fail(ctx, SONAR_E_UNSUPPORTED, "array %dx%d: need nx %% 4 == 0, 4 <= nx <= 64, 1 <= ny <= 64", p->nx, p->ny);
  if (!(p->pitch_m > 0) || !(p->f0_hz > 0) || !(p->bw_hz >= 0) || !(p->pulse_s > 0))
    return fail(ctx, SONAR_E_ARG, "pitch, f0 and pulse must be positive, bw non-negative");
  if (!(p->hfov_rad > 0 && p->hfov_rad < M_PI) || !(p->vfov_rad > 0 && p->vfov_rad < M_PI))
    return fail(ctx, SONAR_E_ARG, "fields of view must lie in (0, pi)");
  if (p->n_beam_az < 1 || p->n_beam_el < 1 || p->n_range < 1)
    return fail(ctx, SONAR_E_ARG, "beam and range counts must be >= 1");
  if ((int64_t)p->n_beam_az * p->n_beam_el > (1 << 24) || p->n_range > (1 << 20))
    return fail(ctx, SONAR_E_UNSUPPORTED, "beam or range count too large");
  if (!(p->r_min_m >= 0) || !(p->r_max_m > p->r_min_m)) return fail(ctx, SONAR_E_ARG, "need 0 <= r_min < r_max");
  if (p->n_ray_az < 1 || p->n_ray_el < 1) return fail(ctx, SONAR_E_ARG, "ray counts must be >= 1");
  if (p->n_sub != 1 && p->n_sub != 4) return fail(ctx, SONAR_E_ARG, "n_sub must be 1 or 4");
  if ((int64_t)p->n_ray_az * p->n_ray_el * p->n_sub > (1 << 29))
    return fail(ctx, SONAR_E_UNSUPPORTED, "too many sub-rays per ping");
  if (p->max_bounces < 0 || p->max_bounces > 3) return fail(ctx, SONAR_E_ARG, "max_bounces must be 0..3");
  if (p->precision < SONAR_FP32 || p->precision > SONAR_FP16) return fail(ctx, SONAR_E_ARG, "unknown precision");
  if (p->thr_mode != 0 && p->thr_mode != 1) return fail(ctx, SONAR_E_ARG, "thr_mode must be 0 or 1");
  if (ssp) {
    if (ssp->n_nodes < 0 || ssp->n_nodes > 2)
      return fail(ctx, SONAR_E_UNSUPPORTED, "sound-speed profiles with %d nodes are not supported", ssp->n_nodes);
    if (ssp->n_nodes > 0 && !ssp->c) return fail(ctx, SONAR_E_ARG, "ssp.c is NULL");
    if (ssp->n_nodes == 2 && (!ssp->z || ssp->z[0] == ssp->z[1]))
      return fail(ctx, SONAR_E_ARG, "ssp nodes need distinct depths");
    for (int i = 0; i < ssp->n_nodes; ++i)
      if (!(ssp->c[i] > 0)) return fail(ctx, SONAR_E_ARG, "ssp speeds must be positive");
  }
  return SONAR_OK;
}

// Rotation matrix of a ping's unit quaternion (w, x, y, z), normalised first, and its
// position (also rounded to FP32 for the FP32 traversal).
// x as an FP32 pair: hi = RN(x), lo = RN(x - hi).
float2 df_pair(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

DevPose dev_pose(const sonar_pose& ps) {
  const double* q = ps.q;
  const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
  DevPose P;
  P.R[0] = 1 - 2 * (y * y + z * z); P.R[1] = 2 * (x * y - w * z);     P.R[2] = 2 * (x * z + w * y);
  P.R[3] = 2 * (x * y + w * z);     P.R[4] = 1 - 2 * (x * x + z * z); P.R[5] = 2 * (y * z - w * x);
  P.R[6] = 2 * (x * z - w * y);     P.R[7] = 2 * (y * z + w * x);     P.R[8] = 1 - 2 * (x * x + y * y);
  for (int k = 0; k < 3; ++k) {
    P.t[k] = ps.t[k];
    P.t32[k] = (float)ps.t[k];
  }
  for (int k = 0; k < 9; ++k) P.R32[k] = (float)P.R[k];
  for (int k = 0; k < 3; ++k) P.t_lo[k] = (float)(P.t[k] - (double)P.t32[k]);
  for (int k = 0; k < 9; ++k) P.R_lo[k] = (float)(P.R[k] - (double)P.R32[k]);
  return P;
}

// c(x, z) of a field, bilinear with positions clamped to the grid (the reference speed
// at the sonar)
double field_c_host(const sonar_field& f, const double* c, double x, double z) {
  double fx = (x - f.x0) / f.dx, fz = (z - f.z0) / f.dz;
  fx = fx < 0.0 ? 0.0 : (fx > f.nx - 1 ? f.nx - 1 : fx);
  fz = fz < 0.0 ? 0.0 : (fz > f.nz - 1 ? f.nz - 1 : fz);
  int i = (int)floor(fx), j = (int)floor(fz);
  if (i > f.nx - 2) i = f.nx - 2;
  if (j > f.nz - 2) j = f.nz - 2;
  const double u = fx - i, v = fz - j;
  return (1.0 - u) * (1.0 - v) * c[j * f.nx + i] + u * (1.0 - v) * c[j * f.nx + i + 1] +
         (1.0 - u) * v * c[(j + 1) * f.nx + i] + u * v * c[(j + 1) * f.nx + i + 1];
}

// The true-time-delay plan (Sec. II.A wide apertures: per-element delays across the
// array). Steering delays x = -U (u_b . p_m) / (c dt) in units of dt / U are linear in
// the element indices, so their extremes over the array sit at its corners; the levels
// floor(x) - 1 .. floor(x) + 2 of every (beam, element) pair span q0 .. q0 + levels - 1.
// The wideband synthesis window covers every row a hit's pulse can reach at any element
// and phase: with the hit's first-tap offset u0 in (-hw, -hw + 1], phase offsets s / U <=
// (U - 1) / U and element delays |e| <= emax = pitch sqrt(cx^2 + cy^2) / (c dt) (the
// largest |u . p_m| / (c dt) over unit directions), row i relative to the first tap is
// reached only for -E1 <= i <= E2.
int derive_ttd(sonar_ctx* ctx, const sonar_params* p, Derived& d) {
  const int U = ctx->ttd_u;
  if (ctx->raw_u > 0) return fail(ctx, SONAR_E_UNSUPPORTED, "true-time delay and raw series are exclusive");
  if (p->precision == SONAR_FP16) return fail(ctx, SONAR_E_UNSUPPORTED, "true-time delay takes the FP32 or BF16 form");
  if (p->nx > 64 || p->ny > 64) return fail(ctx, SONAR_E_UNSUPPORTED, "true-time delay: at most 64 x 64 elements");
  const double cx = 0.5 * (p->nx - 1), cy = 0.5 * (p->ny - 1);
  d.ttd_x_scale = U * p->pitch_m / (d.c_ref * d.dt);
  double xmin = 0.0, xmax = 0.0;
  for (int b = 0; b < p->n_beam_az * p->n_beam_el; ++b) {
    const int bi = b % p->n_beam_az, bj = b / p->n_beam_az;
    const double az = -p->hfov_rad / 2 + (bi + 0.5) * p->hfov_rad / p->n_beam_az;
    const double el = -p->vfov_rad / 2 + (bj + 0.5) * p->vfov_rad / p->n_beam_el;
    const double uy = cos(el) * sin(az), uz = sin(el);
    for (int c = 0; c < 4; ++c) {
      const double ym = (c & 1) ? cx : -cx, zm = (c & 2) ? cy : -cy;
      const double x = -d.ttd_x_scale * (uy * ym + uz * zm);
      xmin = fmin(xmin, x);
      xmax = fmax(xmax, x);
    }
  }
  d.ttd_q0 = (int)floor(xmin) - 1;
  d.ttd_levels = (int)floor(xmax) + 2 - d.ttd_q0 + 1;
  auto floor_div = [](int q, int u) { return (q - (((q % u) + u) % u)) / u; };
  d.ttd_guard = std::max(-floor_div(d.ttd_q0, U), floor_div(d.ttd_q0 + d.ttd_levels - 1, U));
  if (d.ttd_guard > kPad) return fail(ctx, SONAR_E_UNSUPPORTED, "true-time delays span more than %d range samples", kPad);
  const double emax = p->pitch_m * sqrt(cx * cx + cy * cy) / (d.c_ref * d.dt);
  const int E1 = (int)ceil(1.0 + (U - 1.0) / U + emax) - 1;
  const int E2 = (int)ceil(2.0 * d.hw + emax) - 1;
  const int need = E1 + E2 + 1 + 2;  // one row of slack on either side
  d.wb_wt = need <= 12 ? 12 : need <= 16 ? 16 : need <= 20 ? 20 : need <= 24 ? 24 : 0;
  if (!d.wb_wt)
    return fail(ctx, SONAR_E_UNSUPPORTED, "true-time delay: pulse and aperture delays span %d range samples, at most 22",
                need - 2);
  d.wb_e1 = E1 + 1;
  d.wb_f = (128 + U - 1) / U;
  d.wb_uf = U * d.wb_f;
  d.wb_v_lo = -d.hw - d.wb_e1 - emax - 1.0;
  const double v_hi = -d.hw + 1.0 + (d.wb_wt - 1 - d.wb_e1) + (U - 1.0) / U + emax + 1.0;
  d.wb_n_tab = (int)ceil((v_hi - d.wb_v_lo) * d.wb_uf) + 2;
  d.wb_x0 = (-d.wb_e1 - d.wb_v_lo) * d.wb_uf;
  const int64_t smem = (int64_t)d.wb_n_tab * 16 + 32LL * (p->nx + p->ny) * 12 + 256;
  if (smem > 160 * 1024) return fail(ctx, SONAR_E_UNSUPPORTED, "true-time delay: synthesis table too large");
  return SONAR_OK;
}

int derive(sonar_ctx* ctx, const sonar_params* p, const sonar_ssp* ssp, double x_sonar, double z_sonar, int n_pings,
           Derived& d) {
  d.ssp_z0 = 0.0;
  d.ssp_g = 0.0;
  int nn = ssp ? ssp->n_nodes : 0;
  if (nn == 0) {
    if (!(p->c_ref > 0)) return fail(ctx, SONAR_E_ARG, "isovelocity without a profile needs c_ref > 0");
    d.ssp_c0 = p->c_ref;
  } else if (nn == 1) {
    d.ssp_c0 = ssp->c[0];
  } else {
    d.ssp_z0 = ssp->z[0];
    d.ssp_c0 = ssp->c[0];
    d.ssp_g = (ssp->c[1] - ssp->c[0]) / (ssp->z[1] - ssp->z[0]);
  }
  d.curved = d.ssp_g != 0.0;
  d.c_ref = p->c_ref > 0 ? p->c_ref : d.ssp_c0 + d.ssp_g * (z_sonar - d.ssp_z0);
  if (ctx->fld.nx > 0) {
    // the field replaces the profile: rays take the curved-path kernel, the reference
    // speed is c at the sonar unless given
    if (ctx->cross || ctx->vol_n > 0)
      return fail(ctx, SONAR_E_UNSUPPORTED, "a sound-speed field carries no cross terms or volume scatterers");
    d.curved = 1;
    if (!(p->c_ref > 0)) d.c_ref = field_c_host(ctx->fld, ctx->fld_host.data(), x_sonar, z_sonar);
  }
  if (!(d.c_ref > 0)) return fail(ctx, SONAR_E_ARG, "non-positive reference sound speed");
  d.nr = p->n_range;
  d.dr = (p->r_max_m - p->r_min_m) / p->n_range;
  d.dt = 2.0 * d.dr / d.c_ref;
  d.t0 = 2.0 * (p->r_min_m + 0.5 * d.dr) / d.c_ref;
  d.hw = p->pulse_s / d.dt;
  d.taps = (int)floor(2.0 * d.hw) + 1;
  if (ctx->raw_u > 0 && !(d.hw > 2.0))
    return fail(ctx, SONAR_E_UNSUPPORTED, "raw series need a pulse longer than two range samples");
  if (d.taps > 16)
    return fail(ctx, SONAR_E_UNSUPPORTED, "pulse spans %d range samples; at most 16 are supported", d.taps);
  d.T_stop = p->r_max_m / d.c_ref + p->pulse_s / 2.0;
  if (ctx->ttd_u > 0) {
    const int rc = derive_ttd(ctx, p, d);
    if (rc) return rc;
  }
  d.pitch_over_lambda = p->pitch_m * p->f0_hz / d.c_ref;
  d.nr_pad = d.nr + 2 * kPad;
  d.nr_x = (int)round_up(d.nr, 128);
  d.M = p->nx * p->ny;
  d.k_pad = (int)round_up(2LL * d.M, 64);
  d.nb = p->n_beam_az * p->n_beam_el;
  d.n_el = p->n_beam_el;
  d.n_az = p->n_beam_az;
  d.tile_n = ctx->tile_opt != 0   ? ctx->tile_opt
             : ctx->cur_tile_n != 0 ? ctx->cur_tile_n
                                    : pick_tile_n((int64_t)n_pings * d.nr_x / 128, d.nb, ctx->sm_count);
  // Separable beams (Sep1Args): phase-shift beams, a separable taper, BF16 operands (the
  // FP32 and BF16 forms), an array the first stage serves, and an N tile inside one
  // elevation row (the caller's tile wins over the separable form).
  {
    std::vector<double> wx, wy;
    d.sep = ctx->bf_opt == 0 && ctx->ttd_u == 0 && p->precision != SONAR_FP16 && sep1_supported(p->nx, p->ny) &&
            p->n_beam_el * p->ny <= 4096 && taper_separable(p, &wx, &wy);
    if (d.sep && p->n_beam_az % (d.tile_n / 2) != 0) {
      if (ctx->tile_opt != 0) d.sep = 0;
      else if (p->n_beam_az % 128 == 0) d.tile_n = 256;
      else if (p->n_beam_az % 64 == 0) d.tile_n = 128;
      else d.sep = 0;
    }
  }
  d.nb_pad = (int)round_up(d.nb, d.tile_n / 2);
  d.n_phase = p->precision == SONAR_FP32 ? 3 : 1;
  d.n_blank = 0;
  while (d.n_blank < d.nr && p->r_min_m + (d.n_blank + 0.5) * d.dr < p->r_blank_m) ++d.n_blank;
  int np = (isnan(p->surface_z) ? 0 : 1) + (ctx->has_scene ? ctx->sc.n_planes : 0);
  int mb = p->max_bounces > 3 ? 3 : p->max_bounces;
  if (ctx->fld.nx > 0) {
    d.n_routes = 0;  // no eigen-ray search in a field: point scatterers do not echo
  } else if (d.curved) {
    d.n_routes = 1;
  } else {
    int64_t total = 1, cnt = 1;
    for (int len = 1; len <= mb && np > 0; ++len) {
      cnt = len == 1 ? np : cnt * (np - 1);
      total += cnt;
    }
    d.n_routes = (int)total;
  }
  if (d.n_routes > 256) return fail(ctx, SONAR_E_UNSUPPORTED, "too many point-scatterer routes");
  if (ctx->cross && d.curved)
    return fail(ctx, SONAR_E_UNSUPPORTED, "cross-term multipath needs an isovelocity profile");
  if (ctx->vol_n > 0 && d.curved)
    return fail(ctx, SONAR_E_UNSUPPORTED, "volume reverberation needs an isovelocity profile");
  if (ctx->vol_n > 0 && ctx->has_scene && ctx->sc.n_points >= (1 << 21))
    return fail(ctx, SONAR_E_UNSUPPORTED, "volume reverberation keys allow at most 2^21 point scatterers");
  d.wsum = 0.0;
  d.wmax = 0.0;
  for (int m = 0; m < d.M; ++m) {
    double w = p->taper ? (double)p->taper[m] : 1.0;
    if (!(w >= 0)) return fail(ctx, SONAR_E_ARG, "taper weights must be non-negative");
    d.wsum += w;
    d.wmax = fmax(d.wmax, w);
  }
  if (!(d.wsum > 0)) return fail(ctx, SONAR_E_ARG, "taper weights sum to zero");
  d.n_subrays = (int64_t)p->n_ray_az * p->n_ray_el * p->n_sub;
  int64_t npts = ctx->has_scene ? ctx->sc.n_points : 0;
  if (ctx->cross && (d.n_subrays > (1LL << 27) || npts > 16384))
    return fail(ctx, SONAR_E_UNSUPPORTED, "cross-term keys hold at most 2^27 sub-rays and 16384 points");
  // a route emits one hit per segment; with cross terms every segment after a
  // reflection adds two, and a point's routes pair up in every ordered combination
  d.hit_cap_per_ping = ctx->cross ? d.n_subrays * (1 + 3 * (int64_t)p->max_bounces) + npts * d.n_routes * d.n_routes
                                  : d.n_subrays * (1 + p->max_bounces) + npts * d.n_routes;
  d.hit_cap_per_ping += ctx->vol_n;
  return SONAR_OK;
}

uint32_t seed32(uint64_t s) { return (uint32_t)(s ^ (s >> 32)); }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

// box_k: K elements per box row, 64 (128-byte swizzle) or 32 (64-byte swizzle).
int make_map(sonar_ctx* ctx, CUtensorMap* m, void* base, int64_t rows, int64_t cols, int box_rows, bool f16,
             int box_k = 64) {
  auto fn = encode_fn();
  if (!fn) return fail(ctx, SONAR_E_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  box_k == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, SONAR_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return SONAR_OK;
}

// (Re)build ray table, pulse table and steering matrix when their parameters change.
template <typename T>
int grow(sonar_ctx* ctx, T*& ptr, int64_t& cap, int64_t need, size_t elem, bool zero);

// Extra synthesis cost of a non-empty range row, in units of one hit, for the
// cost-balanced split of the sorted hits over the persistent synthesis CTAs.
#ifndef SONAR_SYNTH_ROW_COST
#define SONAR_SYNTH_ROW_COST 16
#endif
constexpr int kSynthRowCost = SONAR_SYNTH_ROW_COST;

// Water-column scatterers up to this count are processed in the Morton order of their
// positions (a host sort at the first ping with a new count or seed); beyond it, in index
// order.
constexpr int64_t kVolSortMax = 1LL << 24;

// 10-bit value spread to every third bit (Morton interleave).
uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x3FFu;
  x = (x | x << 16) & 0x30000FFull;
  x = (x | x << 8) & 0x300F00Full;
  x = (x | x << 4) & 0x30C30C3ull;
  x = (x | x << 2) & 0x9249249ull;
  return x;
}

int ensure_tables(sonar_ctx* ctx, const sonar_params* p, const Derived& d) {
  if (ctx->vol_n > 0 && ctx->vol_n <= kVolSortMax) {
    // the scatterer positions are lo + (hi - lo) u with u from the hash words: their top
    // 10 bits per axis give the Morton key, whatever the box
    const uint32_t s32 = seed32(p->seed);
    std::vector<uint8_t> kv;
    key_add(kv, ctx->vol_n); key_add(kv, s32);
    if (kv != ctx->vol_key || !ctx->vol_order) {
      const int64_t n = ctx->vol_n;
      std::vector<uint64_t> key((size_t)n);
      for (int64_t i = 0; i < n; ++i) {
        uint32_t x = (uint32_t)i, y = (uint32_t)((uint64_t)i >> 32), z = 0x564F4Cu, w = s32;
        pcg4d(x, y, z, w);
        key[(size_t)i] = ((spread3(x >> 22) | spread3(y >> 22) << 1 | spread3(z >> 22) << 2) << 32) | (uint64_t)i;
      }
      std::sort(key.begin(), key.end());
      std::vector<int32_t> ord((size_t)n);
      for (int64_t j = 0; j < n; ++j) ord[(size_t)j] = (int32_t)(key[(size_t)j] & 0xFFFFFFFFull);
      int rc;
      if ((rc = grow(ctx, ctx->vol_order, ctx->vol_order_cap, n, sizeof(int32_t), false))) return rc;
      CU(cudaMemcpy(ctx->vol_order, ord.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice));
      ctx->vol_key = kv;
    }
  }
  std::vector<uint8_t> k;
  key_add(k, p->n_ray_az); key_add(k, p->n_ray_el); key_add(k, p->n_sub);
  key_add(k, p->hfov_rad); key_add(k, p->vfov_rad); key_add(k, p->seed);
  if (k != ctx->ray_key) {
    dfree(ctx->ray_dirs);
    dfree(ctx->ray_dirs32);
    dfree(ctx->row_domega);
    CU(cudaMalloc(&ctx->ray_dirs, sizeof(double) * 3 * d.n_subrays));
    CU(cudaMalloc(&ctx->ray_dirs32, sizeof(float) * 6 * d.n_subrays));
    CU(cudaMalloc(&ctx->row_domega, sizeof(float) * p->n_ray_el));
    CU(launch_ray_table(ctx->ray_dirs, ctx->ray_dirs32, ctx->row_domega, p->n_ray_az, p->n_ray_el, p->n_sub,
                        p->hfov_rad, p->vfov_rad, seed32(p->seed), ctx->stream));
    ctx->ray_key = k;
  }
  k.clear();
  key_add(k, p->pulse_s); key_add(k, p->bw_hz);
  if (k != ctx->rtab_key) {
    if (!ctx->rtab) CU(cudaMalloc(&ctx->rtab, sizeof(float2) * (kRTab + 1 + kRTabS + 5)));
    CU(launch_rtab(ctx->rtab, ctx->rtab + kRTab + 1, p->pulse_s, p->bw_hz, ctx->stream));
    ctx->rtab_key = k;
  }
  if (ctx->raw_u > 0) {
    // raw series: the pulse shifted by s dt / U on both table grids, and the matched
    // filter's taps over |d| <= D range samples
    const int D = (int)ceil(p->pulse_s / (2.0 * d.dt)) + 1;
    k.clear();
    key_add(k, p->pulse_s); key_add(k, p->bw_hz); key_add(k, d.dt); key_add(k, ctx->raw_u);
    if (k != ctx->ptab_key) {
      dfree(ctx->ptab);
      const int64_t n = (int64_t)ctx->raw_u * (kRTab + 1 + kRTabS + 5 + 2 * D + 1);
      CU(cudaMalloc(&ctx->ptab, sizeof(float2) * n));
      float2* big = ctx->ptab;
      float2* small = big + (int64_t)ctx->raw_u * (kRTab + 1);
      float2* taps = small + (int64_t)ctx->raw_u * (kRTabS + 5);
      CU(launch_ptab(big, small, taps, ctx->raw_u, D, p->pulse_s, p->bw_hz, d.dt, ctx->stream));
      ctx->ptab_u = ctx->raw_u;
      ctx->ptab_d = D;
      ctx->ptab_key = k;
    }
  }
  if (ctx->ttd_u > 0) {
    k.clear();
    key_add(k, p->pulse_s); key_add(k, p->bw_hz); key_add(k, d.dt); key_add(k, d.wb_v_lo); key_add(k, d.wb_uf);
    key_add(k, d.wb_n_tab);
    if (k != ctx->wtab_key) {
      dfree(ctx->wtab);
      CU(cudaMalloc(&ctx->wtab, sizeof(float4) * d.wb_n_tab));
      CU(launch_wtab(ctx->wtab, d.wb_n_tab, d.wb_v_lo, 1.0 / d.wb_uf, d.dt, p->pulse_s, p->bw_hz, ctx->stream));
      ctx->wtab_key = k;
    }
  }
  k.clear();
  key_add(k, p->nx); key_add(k, p->ny); key_add(k, d.pitch_over_lambda); key_add(k, p->hfov_rad);
  key_add(k, p->vfov_rad); key_add(k, p->n_beam_az); key_add(k, p->n_beam_el); key_add(k, p->precision);
  key_add(k, d.tile_n); key_add(k, ctx->ttd_u); key_add(k, d.ttd_q0); key_add(k, d.ttd_levels);
  key_add(k, d.ttd_x_scale);
  for (int m = 0; m < d.M; ++m) key_add(k, p->taper ? p->taper[m] : 1.0f);
  // beam-centre direction cosines (u_y, u_z), FP64, for either steering operand
  auto upload_uyz = [&]() -> int {
    std::vector<double2> uyz((size_t)d.nb);
    for (int b = 0; b < d.nb; ++b) {
      const int bi = b % p->n_beam_az, bj = b / p->n_beam_az;
      const double az = -p->hfov_rad / 2 + (bi + 0.5) * p->hfov_rad / p->n_beam_az;
      const double el = -p->vfov_rad / 2 + (bj + 0.5) * p->vfov_rad / p->n_beam_el;
      uyz[(size_t)b] = make_double2(cos(el) * sin(az), sin(el));
    }
    int rc;
    if ((rc = grow(ctx, ctx->beam_uyz, ctx->beam_uyz_cap, d.nb, sizeof(double2), false))) return rc;
    CU(cudaMemcpyAsync(ctx->beam_uyz, uyz.data(), sizeof(double2) * d.nb, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));  // the host table is released on return
    return SONAR_OK;
  };
  if (d.sep) {
    // separable beams: Fz[el][my] = wy[my] exp(-j 2 pi (d / lambda) (my - (ny-1)/2) sin el)
    // (FP64 phase reduced modulo one cycle), and the second stage's steering operand: the
    // steering matrix of one array row with taper wx, the full taper's sum as divisor
    if (k != ctx->sep_key) {
      std::vector<double> wx, wy;
      taper_separable(p, &wx, &wy);
      std::vector<float2> fz((size_t)p->n_beam_el * p->ny);
      for (int j = 0; j < p->n_beam_el; ++j) {
        const double el = -p->vfov_rad / 2 + (j + 0.5) * p->vfov_rad / p->n_beam_el, uz = sin(el);
        for (int my = 0; my < p->ny; ++my) {
          const double cyc = d.pitch_over_lambda * (my - 0.5 * (p->ny - 1)) * uz;
          const double ph = 2.0 * kPi * (cyc - floor(cyc));
          fz[(size_t)j * p->ny + my] = make_float2((float)(wy[(size_t)my] * cos(ph)), (float)(-wy[(size_t)my] * sin(ph)));
        }
      }
      int rc;
      if ((rc = grow(ctx, ctx->sep_fz, ctx->sep_fz_cap, (int64_t)fz.size(), sizeof(float2), false))) return rc;
      CU(cudaMemcpyAsync(ctx->sep_fz, fz.data(), sizeof(float2) * fz.size(), cudaMemcpyHostToDevice, ctx->stream));
      std::vector<float> wxf(wx.begin(), wx.end());
      dfree(ctx->taper_x_dev);
      CU(cudaMalloc(&ctx->taper_x_dev, sizeof(float) * p->nx));
      CU(cudaMemcpyAsync(ctx->taper_x_dev, wxf.data(), sizeof(float) * p->nx, cudaMemcpyHostToDevice, ctx->stream));
      const size_t elems = (size_t)2 * d.nb_pad * 64;
      if (elems != ctx->ysep_elems) {
        dfree(ctx->ysep_hi);
        dfree(ctx->ysep_lo);
        CU(cudaMalloc(&ctx->ysep_hi, elems * 2));
        CU(cudaMalloc(&ctx->ysep_lo, elems * 2));
        ctx->ysep_elems = elems;
      }
      if ((rc = upload_uyz())) return rc;  // also waits for the Fz and taper copies
      double wxmax = 0.0;
      for (double v : wx) wxmax = fmax(wxmax, v);
      ctx->ysep_gain = d.wsum / wxmax;  // steering entries scaled to at most 1
      SteerArgs sa;
      sa.beam_uyz = ctx->beam_uyz;
      sa.nx = p->nx; sa.ny = 1; sa.n_beam_az = p->n_beam_az; sa.n_beam_el = p->n_beam_el;
      sa.nb_pad = d.nb_pad; sa.k_pad = 64; sa.hfov = p->hfov_rad; sa.vfov = p->vfov_rad;
      sa.pitch_over_lambda = d.pitch_over_lambda; sa.taper = ctx->taper_x_dev; sa.wsum = d.wsum;
      sa.gain = ctx->ysep_gain; sa.mode = p->precision; sa.y_hi = ctx->ysep_hi; sa.y_lo = ctx->ysep_lo;
      sa.n_levels = 1; sa.q0 = 0; sa.ttd = 0; sa.x_scale = 0.0;
      CU(launch_steer(sa, ctx->stream));
      ctx->sep_key = k;
    }
    return SONAR_OK;
  }
  if (k != ctx->steer_key) {
    size_t elems = (size_t)2 * d.nb_pad * d.k_pad * d.ttd_levels;
    if (elems != ctx->y_elems) {
      dfree(ctx->y_hi);
      dfree(ctx->y_lo);
      CU(cudaMalloc(&ctx->y_hi, elems * 2));
      CU(cudaMalloc(&ctx->y_lo, elems * 2));
      ctx->y_elems = elems;
    }
    dfree(ctx->taper_dev);
    if (p->taper) {
      CU(cudaMalloc(&ctx->taper_dev, sizeof(float) * d.M));
      CU(cudaMemcpyAsync(ctx->taper_dev, p->taper, sizeof(float) * d.M, cudaMemcpyHostToDevice, ctx->stream));
    }
    ctx->y_gain = d.wsum / d.wmax;  // steering entries scaled to at most 1
    int rc;
    if ((rc = upload_uyz())) return rc;
    SteerArgs sa;
    sa.beam_uyz = ctx->beam_uyz;
    sa.nx = p->nx; sa.ny = p->ny; sa.n_beam_az = p->n_beam_az; sa.n_beam_el = p->n_beam_el;
    sa.nb_pad = d.nb_pad; sa.k_pad = d.k_pad; sa.hfov = p->hfov_rad; sa.vfov = p->vfov_rad;
    sa.pitch_over_lambda = d.pitch_over_lambda; sa.taper = ctx->taper_dev; sa.wsum = d.wsum;
    sa.gain = ctx->y_gain; sa.mode = p->precision; sa.y_hi = ctx->y_hi; sa.y_lo = ctx->y_lo;
    sa.n_levels = d.ttd_levels; sa.q0 = d.ttd_q0; sa.ttd = ctx->ttd_u > 0; sa.x_scale = d.ttd_x_scale;
    CU(launch_steer(sa, ctx->stream));
    ctx->steer_key = k;
  }
  return SONAR_OK;
}

template <typename T>
int grow(sonar_ctx* ctx, T*& ptr, int64_t& cap, int64_t need, size_t elem, bool zero) {
  if (need <= cap && ptr) return SONAR_OK;
  dfree(ptr);
  cudaError_t e = cudaMalloc((void**)&ptr, (size_t)need * elem);
  if (e != cudaSuccess) {
    cap = 0;
    return fail(ctx, SONAR_E_NOMEM, "cudaMalloc of %lld bytes failed: %s", (long long)(need * elem), cudaGetErrorString(e));
  }
  if (zero) CU(cudaMemsetAsync(ptr, 0, (size_t)need * elem, ctx->stream));
  cap = need;
  return SONAR_OK;
}

int ensure_workspace(sonar_ctx* ctx, int P, const Derived& d) {
  int rc;
  if (P > ctx->p_cap) {
    if (ctx->pose_host) cudaFreeHost(ctx->pose_host);
    if (ctx->n_cloud_host) cudaFreeHost(ctx->n_cloud_host);
    ctx->pose_host = nullptr;
    ctx->n_cloud_host = nullptr;
    dfree(ctx->poses); dfree(ctx->gain); dfree(ctx->pmax); dfree(ctx->n_cloud_dev);
    CU(cudaMallocHost(&ctx->pose_host, sizeof(DevPose) * P));
    CU(cudaHostGetDevicePointer((void**)&ctx->pose_map, ctx->pose_host, 0));
    CU(cudaMallocHost(&ctx->n_cloud_host, sizeof(long long) * P));
    CU(cudaHostGetDevicePointer((void**)&ctx->n_cloud_map, ctx->n_cloud_host, 0));
    CU(cudaMalloc(&ctx->poses, sizeof(DevPose) * P));
    CU(cudaMalloc(&ctx->gain, sizeof(float) * P));
    CU(cudaMalloc(&ctx->pmax, sizeof(unsigned) * P));
    CU(cudaMalloc(&ctx->n_cloud_dev, sizeof(long long) * P));
    ctx->p_cap = P;
  }
  if (!ctx->n_hits) CU(cudaMalloc(&ctx->n_hits, 2 * sizeof(unsigned long long)));
  if (!ctx->err_dev) CU(cudaMalloc(&ctx->err_dev, sizeof(int)));
  if (!ctx->synth_bounds) CU(cudaMalloc(&ctx->synth_bounds, sizeof(int32_t) * (ctx->sm_count + 1)));
  int64_t hit_need = (int64_t)P * d.hit_cap_per_ping;
  if (hit_need < 1) hit_need = 1;
  if (hit_need > ctx->ws_hits || !ctx->hits) {
    int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    dfree(ctx->hits); dfree(ctx->sorted); dfree(ctx->dbg_tau); dfree(ctx->sorted_n); dfree(ctx->rank);
    if ((rc = grow(ctx, ctx->sorted_n, c3, hit_need, sizeof(int32_t), false))) return rc;
    int64_t c4 = 0;
    if ((rc = grow(ctx, ctx->rank, c4, hit_need, sizeof(int32_t), false))) return rc;
    if ((rc = grow(ctx, ctx->hits, c0, hit_need, sizeof(HitRec), false))) return rc;
    if ((rc = grow(ctx, ctx->sorted, c1, hit_need, sizeof(HitRec), false))) return rc;
    if ((rc = grow(ctx, ctx->dbg_tau, c2, hit_need, sizeof(double), false))) return rc;
    ctx->ws_hits = hit_need;
  }
  ctx->hit_cap = hit_need;
  const int64_t pt_need = ctx->cross ? (int64_t)P * (ctx->has_scene ? ctx->sc.n_points : 0) * d.n_routes : 0;
  if (pt_need > ctx->ws_pt_route) {
    int64_t c0 = 0;
    dfree(ctx->pt_route);
    if ((rc = grow(ctx, ctx->pt_route, c0, pt_need, sizeof(PtRoute), false))) return rc;
    ctx->ws_pt_route = pt_need;
  }
  int64_t bins = (int64_t)P * d.nr_pad + 1;
  if (bins > ctx->ws_bins || !ctx->counts) {
    int64_t c0 = 0, c1 = 0;
    dfree(ctx->counts); dfree(ctx->offsets);
    if ((rc = grow(ctx, ctx->counts, c0, bins, sizeof(int32_t), false))) return rc;
    if ((rc = grow(ctx, ctx->offsets, c1, bins, sizeof(int32_t), false))) return rc;
    ctx->ws_bins = bins;
  }
  // guard rows: taps past the last ping and whole tensor-core tiles (up to 96 rows)
  int64_t s_need = ((int64_t)P * d.nr_pad + 2 * kPad + 96) * d.M;
  if (s_need > ctx->ws_s || !ctx->S) {
    int64_t c0 = 0;
    dfree(ctx->S);
    if ((rc = grow(ctx, ctx->S, c0, s_need, sizeof(float2), false))) return rc;
    ctx->ws_s = s_need;
  }
  ctx->s_elems = s_need;
  const int phases = ctx->raw_u > 0 ? ctx->raw_u : ctx->ttd_u;
  if (phases > 0 && (s_need * phases > ctx->ws_raw || !ctx->S_raw)) {
    int64_t c0 = 0;
    dfree(ctx->S_raw);
    if ((rc = grow(ctx, ctx->S_raw, c0, s_need * phases, sizeof(float2), false))) return rc;
    ctx->ws_raw = s_need * phases;
  }
  // true-time delay: the echo operand holds every phase, each ping's rows with guard rows
  // on either side for the level offsets
  // separable beams: one block of P nr_x rows of 64 columns per elevation row
  int64_t x_need = ctx->ttd_u > 0 ? (int64_t)ctx->ttd_u * P * (d.nr_x + 2 * d.ttd_guard) * d.k_pad
                   : d.sep        ? (int64_t)d.n_el * P * d.nr_x * 64
                                  : (int64_t)P * d.nr_x * d.k_pad;
  if (x_need != ctx->ws_x || !ctx->x_hi) {
    int64_t c0 = 0, c1 = 0;
    dfree(ctx->x_hi); dfree(ctx->x_lo);
    if ((rc = grow(ctx, ctx->x_hi, c0, x_need, 2, true))) return rc;
    if ((rc = grow(ctx, ctx->x_lo, c1, x_need, 2, true))) return rc;
    ctx->ws_x = x_need;
  }
  ctx->x_elems = x_need;
  int64_t keys_need = (int64_t)P * d.nb;
  if (!ctx->keys || keys_need > ctx->keys_cap) {
    dfree(ctx->keys);
    CU(cudaMalloc(&ctx->keys, sizeof(unsigned long long) * keys_need));
    ctx->keys_cap = keys_need;
  }
  return SONAR_OK;
}

// Where an output lives: device memory (written in place), pinned host memory mapped
// into this device's address space (written in place through the mapping, so results
// cross to the host while the kernels run), or other host memory (staged on the
// device and copied at the end). *dev is the address the kernels write to.
enum class Mem { Device, Mapped, Host };
Mem classify(void* p, void** dev) {
  *dev = nullptr;
  if (!p) return Mem::Host;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return Mem::Host;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    *dev = p;
    return Mem::Device;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *dev = at.devicePointer;
    return Mem::Mapped;
  }
  return Mem::Host;
}

struct Outputs {
  float* env;               // where the kernels write
  sonar_point* cloud;
  int64_t cap;
  float* env_host;          // staged outputs copied back in the pipeline: the caller's host
  sonar_point* cloud_host;  // buffers, else nullptr
  int64_t env_elems;
  const DevPose* pose_src;              // device mapping of the pinned poses the first kernel reads
  long long* n_cloud_map;               // device mappings of the pinned per-ping point
  unsigned long long* counters_map;     // counts and of the hit count / error words
};

// Arguments of the ray-casting kernels for P pings with parameters p (derived values d).
TraceArgs trace_args(const sonar_ctx* ctx, int P, const sonar_params* p, const Derived& d, bool pairs) {
  TraceArgs ta;
  memset(&ta, 0, sizeof(ta));
  ta.sc = ctx->sc;
  ta.poses = ctx->poses;
  ta.ray_dirs = ctx->ray_dirs;
  ta.ray_dirs32 = ctx->ray_dirs32;
  ta.ray_dirs_lo = ctx->ray_dirs32 + 3 * d.n_subrays;
  ta.row_domega = ctx->row_domega;
  ta.n_pings = P;
  ta.n_ray_az = p->n_ray_az;
  ta.n_ray_el = p->n_ray_el;
  ta.n_sub = p->n_sub;
  ta.n_subrays = (int32_t)d.n_subrays;
  ta.max_bounces = p->max_bounces;
  ta.has_surface = isnan(p->surface_z) ? 0 : 1;
  ta.curved = d.curved;
  ta.surface_z = p->surface_z;
  ta.r_surface = p->r_surface;
  ta.r_seabed = p->r_seabed;
  ta.alpha = p->alpha_np_per_m;
  ta.alpha32 = (float)p->alpha_np_per_m;
  ta.seed32 = seed32(p->seed);
  ta.ssp_z0 = d.ssp_z0;
  ta.ssp_c0 = d.ssp_c0;
  ta.ssp_g = d.ssp_g;
  ta.inv_c0 = 1.0 / d.ssp_c0;
  ta.two_inv_c0 = 2.0 * ta.inv_c0;
  ta.T_stop = d.T_stop;
  ta.L_stop = d.T_stop * d.ssp_c0;
  ta.L_stop32 = (float)ta.L_stop;
  ta.surface_z32 = (float)p->surface_z;
  ta.t0 = d.t0;
  ta.inv_dt = 1.0 / d.dt;
  ta.t0_dt = d.t0 * ta.inv_dt;
  ta.hw = d.hw;
  ta.f0 = p->f0_hz;
  ta.L_stop_df = df_pair(ta.L_stop);
  ta.surface_z_df = df_pair(isnan(p->surface_z) ? 0.0 : p->surface_z);
  ta.two_inv_c0_df = df_pair(ta.two_inv_c0);
  ta.f0_df = df_pair(ta.f0);
  ta.inv_dt_df = df_pair(ta.inv_dt);
  ta.t0_dt_df = df_pair(ta.t0_dt);
  ta.hw_df = df_pair(ta.hw);
  ta.nr_pad = d.nr_pad;
  ta.n_routes = d.n_routes;
  ta.cross = ctx->cross;
  ta.warp_walk = ctx->traversal;
  ta.pt_route = pairs ? ctx->pt_route : nullptr;
  ta.vol_n = ctx->vol_n;
  for (int k = 0; k < 3; ++k) {
    ta.vol_lo[k] = ctx->vol_lo[k];
    ta.vol_hi[k] = ctx->vol_hi[k];
    ta.vol_lo_df[k] = df_pair(ctx->vol_lo[k]);
    ta.vol_span_df[k] = df_pair(ctx->vol_hi[k] - ctx->vol_lo[k]);
  }
  ta.vol_sigma = ctx->vol_sigma;
  ta.fld_nx = ctx->fld.nx;
  ta.fld_nz = ctx->fld.nz;
  ta.fld_x0 = ctx->fld.x0;
  ta.fld_dx = ctx->fld.dx;
  ta.fld_z0 = ctx->fld.z0;
  ta.fld_dz = ctx->fld.dz;
  ta.fld_h = ctx->fld.step_m;
  ta.fld_idx = ctx->fld.nx > 0 ? 1.0 / ctx->fld.dx : 0.0;
  ta.fld_idz = ctx->fld.nx > 0 ? 1.0 / ctx->fld.dz : 0.0;
  ta.fld_c = ctx->fld_c;
  ta.vol_order = ctx->vol_n > 0 && ctx->vol_n <= kVolSortMax ? ctx->vol_order : nullptr;
  ta.hits = ctx->hits;
  ta.bin_rank = ctx->rank;
  ta.bin_counts = ctx->counts;
  ta.dbg_tau = ctx->debug ? ctx->dbg_tau : nullptr;
  ta.n_hits = ctx->n_hits;
  ta.hit_cap = ctx->hit_cap;
  ta.err = ctx->err_dev;
  return ta;
}

// CTAs per cluster of the beamforming contraction over tiles_m row tiles: the library's
// choice, or the option's size where it fits.
int gemm_cluster_for(const sonar_ctx* ctx, int tiles_m, const Derived& d) {
  if (ctx->gemm_cluster > 0)
    return gemm_cluster_fits(ctx->gemm_cluster, tiles_m, d.tile_n, d.n_phase) ? ctx->gemm_cluster : 1;
  // Separable second stage: K = 2 nx is one K block per tile, so sharing the B tile by
  // multicast saves little while the CTA pair's lockstep on every stage costs more (C2:
  // 0.0205 ms in clusters of two, 0.0192 ms without).
  if (d.sep) return 1;
  return gemm_cluster_size(tiles_m, d.tile_n, d.n_phase, ctx->sm_count);
}

// Enqueue the whole pipeline for P pings on the context stream (graph-capturable:
// no host synchronisation, fixed grids that read device-side counts).
int enqueue(sonar_ctx* ctx, int P, const sonar_params* p, const Derived& d, const Outputs& o, int* kernels) {
  cudaStream_t st = ctx->stream;
  // stage boundaries: 0 trace 1 bin 2 synth 3 convert 4 beamform 5 peaks 6
  auto mark = [&](int i) {
    if (ctx->timing) cudaEventRecord(ctx->stage_ev[i], st);
  };
  const bool fp16 = p->precision == SONAR_FP16;
  // clear, trace, scan, scatter, synthesis, convert, GEMM, peaks; points (and their cross
  // pairs); FP16 absmax and gain; raw phases
  const bool pairs = ctx->cross && ctx->sc.n_points > 0;
  *kernels = 8 + (ctx->sc.n_points > 0 ? 1 : 0) + (pairs ? 1 : 0) + (ctx->vol_n > 0 ? 1 : 0) + (fp16 ? 2 : 0) +
             (ctx->raw_u > 0 ? ctx->raw_u : 0);
  // the poses the host has just written into the pinned staging record
  mark(0);
  // every buffer that starts at zero is cleared up front, in one launch, so the kernels
  // run back to back
  const int32_t n_bins = P * d.nr_pad;
  const int phases = ctx->raw_u > 0 ? ctx->raw_u : ctx->ttd_u;
  k_clear<<<4 * ctx->sm_count, 256, 0, st>>>(ctx->S, ctx->s_elems, phases > 0 ? ctx->S_raw : nullptr,
                                             ctx->s_elems * phases, ctx->counts, n_bins, ctx->keys,
                                             (int64_t)P * d.nb, ctx->pmax, P, ctx->n_hits, ctx->err_dev,
                                             reinterpret_cast<const uint4*>(o.pose_src),
                                             reinterpret_cast<uint4*>(ctx->poses), (int)(sizeof(DevPose) / 16) * P);
  CU(cudaGetLastError());
  TraceArgs ta = trace_args(ctx, P, p, d, pairs);
  CU(launch_trace(ta, ctx->sm_count, st));
  CU(launch_points(ta, st));
  if (pairs) CU(launch_point_pairs(ta, st));
  CU(launch_volume(ta, st));
  mark(1);
  CU(launch_bin(ctx->hits, ctx->n_hits, n_bins, ctx->counts, ctx->offsets, ctx->rank, ctx->sorted, ctx->sorted_n, ctx->sm_count,
                ctx->synth_bounds, ctx->sm_count, kSynthRowCost, st));
  mark(2);
  SynthArgs sa;
  sa.hits_sorted = ctx->sorted;
  sa.sorted_n = ctx->sorted_n;
  sa.n_valid = ctx->offsets + n_bins;
  sa.bounds = ctx->synth_bounds;  // persistent synthesis kernels run one CTA per SM
  sa.rtab = ctx->rtab;
  sa.rtab_scale = (float)(d.dt * kRTab / (2.0 * p->pulse_s));
  sa.rtab_s = ctx->rtab + kRTab + 1;
  sa.cplx_taps = 0;
  sa.rtab_s_scale = (float)(d.dt * kRTabS / (2.0 * p->pulse_s));
  sa.taps = d.taps;
  sa.nx = p->nx;
  sa.ny = p->ny;
  sa.pitch_over_lambda = (float)d.pitch_over_lambda;
  sa.S = ctx->S;
  sa.total_rows = (int64_t)P * d.nr_pad;
  sa.n_pass = p->precision == SONAR_FP32 ? 3 : 1;
  sa.mma_flop = ctx->n_hits + 1;
  sa.err = ctx->err_dev;
  static const int kPairs[5] = {0, 0, 32, 64, 96};
  const bool tc = ctx->synth_opt != 1 && synth_tc_supported(p->nx, p->ny, d.taps);
  const int want_pairs = ctx->synth_opt >= 2 ? kPairs[ctx->synth_opt] : ctx->cur_pairs;
  if (ctx->ttd_u > 0) {
    // wideband echoes at the U phases, the element delays kept in the envelope
    SynthWbArgs wa;
    wa.hits_sorted = ctx->sorted;
    wa.n_valid = ctx->offsets + n_bins;
    wa.tab = ctx->wtab;
    wa.n_tab = d.wb_n_tab;
    wa.uf = d.wb_uf;
    wa.f = d.wb_f;
    wa.tab_x0 = (float)d.wb_x0;
    wa.e1 = d.wb_e1;
    wa.n_phases = ctx->ttd_u;
    wa.nx = p->nx;
    wa.ny = p->ny;
    wa.pitch_over_lambda = (float)d.pitch_over_lambda;
    wa.pitch_uf = (float)(p->pitch_m / (d.c_ref * d.dt) * d.wb_uf);
    wa.S = ctx->S_raw;
    wa.phase_stride = ctx->s_elems;
    wa.total_rows = (int64_t)P * d.nr_pad;
    wa.err = ctx->err_dev;
    CU(launch_synth_wb(wa, d.wb_wt, ctx->sm_count, st));
  } else if (ctx->raw_u == 0) {
    if (tc) CU(launch_synth_tc(sa, want_pairs, ctx->sm_count, st));
    else CU(launch_synth(sa, ctx->sm_count, st));
  } else {
    // raw series: one synthesis pass per phase s with the pulse shifted by s dt / U in
    // place of its autocorrelation (the same hits, sorted by the same rows), then the
    // matched filter into S
    const int U = ctx->raw_u;
    for (int s = 0; s < U; ++s) {
      SynthArgs sr = sa;
      sr.rtab = ctx->ptab + (int64_t)s * (kRTab + 1);
      sr.rtab_s = ctx->ptab + (int64_t)U * (kRTab + 1) + (int64_t)s * (kRTabS + 5);
      sr.cplx_taps = 1;
      sr.S = ctx->S_raw + (int64_t)s * ctx->s_elems;
      if (tc) CU(launch_synth_tc(sr, want_pairs, ctx->sm_count, st));
      else CU(launch_synth(sr, ctx->sm_count, st));
    }
    MfArgs ma;
    ma.raw = ctx->S_raw;
    ma.phase_stride = ctx->s_elems;
    ma.S = ctx->S;
    ma.taps = ctx->ptab + (int64_t)U * (kRTab + 1 + kRTabS + 5);
    ma.U = U;
    ma.D = ctx->ptab_d;
    ma.nr = d.nr;
    ma.nr_pad = d.nr_pad;
    ma.M = d.M;
    ma.n_pings = P;
    CU(launch_mfilter(ma, st));
  }
  mark(3);
  const bool ttd = ctx->ttd_u > 0;
  const int x_rows = ttd ? d.nr_x + 2 * d.ttd_guard : d.nr_x;
  ConvertArgs ca;
  ca.S = ttd ? ctx->S_raw : ctx->S;
  ca.phase_stride = ttd ? ctx->s_elems : 0;
  ca.n_phases = ttd ? ctx->ttd_u : 1;
  ca.x_rows = x_rows;
  ca.x_guard = ttd ? d.ttd_guard : 0;
  ca.n_pings = P;
  ca.nr = d.nr;
  ca.nr_pad = d.nr_pad;
  ca.nr_x = d.nr_x;
  ca.M = d.M;
  ca.k_pad = d.k_pad;
  ca.mode = p->precision;
  ca.gain = ctx->gain;
  ca.x_hi = ctx->x_hi;
  ca.x_lo = ctx->x_lo;
  if (d.sep) {
    // separable beams, first stage: the echoes summed over the array's rows per elevation
    Sep1Args s1;
    s1.S = ctx->S;
    s1.fz = ctx->sep_fz;
    s1.n_pings = P;
    s1.nr = d.nr;
    s1.nr_pad = d.nr_pad;
    s1.nr_x = d.nr_x;
    s1.nx = p->nx;
    s1.ny = p->ny;
    s1.n_el = d.n_el;
    s1.k_pad = 64;
    s1.mode = p->precision;
    s1.x_hi = ctx->x_hi;
    s1.x_lo = ctx->x_lo;
    s1.err = ctx->err_dev;
    CU(launch_sep1(s1, ctx->sm_count, st));
  } else {
    CU(launch_convert(ca, ctx->sm_count, st));
  }
  mark(4);
  GemmArgs ga;
  memset(&ga, 0, sizeof(ga));
  const bool f16 = fp16;
  int rc;
  const int box_k = d.n_phase == 3 ? 32 : 64;
  // separable beams: the second stage reads K = 64 (one array row, re and im) from the
  // tile's elevation block of the first stage's output
  const int64_t x_cols = d.sep ? 64 : d.k_pad;
  const int64_t x_map_rows = d.sep ? (int64_t)d.n_el * P * x_rows : (int64_t)ca.n_phases * P * x_rows;
  const int64_t y_cols = d.sep ? 64 : (int64_t)d.k_pad * d.ttd_levels;
  void* const yh = d.sep ? ctx->ysep_hi : ctx->y_hi;
  void* const yl = d.sep ? ctx->ysep_lo : ctx->y_lo;
  if ((rc = make_map(ctx, &ga.map_xh, ctx->x_hi, x_map_rows, x_cols, 128, f16, box_k))) return rc;
  if ((rc = make_map(ctx, &ga.map_xl, ctx->x_lo, x_map_rows, x_cols, 128, f16, box_k))) return rc;
  ga.tiles_m = P * d.nr_x / 128;
  // clusters of CTAs load a share of each B tile apiece and multicast it
  ga.cluster = gemm_cluster_for(ctx, ga.tiles_m, d);
  const int y_box = d.tile_n / ga.cluster;
  if ((rc = make_map(ctx, &ga.map_yh, yh, 2LL * d.nb_pad, y_cols, y_box, f16, box_k))) return rc;
  if ((rc = make_map(ctx, &ga.map_yl, yl, 2LL * d.nb_pad, y_cols, y_box, f16, box_k))) return rc;
  ga.tiles_n = 2 * d.nb_pad / d.tile_n;
  ga.k_blocks = (int)(y_cols / 64);
  ga.x_kpad = (int)x_cols;
  ga.sep_az = d.sep ? d.n_az : 0;
  ga.x_el_rows = (int64_t)P * x_rows;
  ga.ttd_u = ctx->ttd_u;
  ga.ttd_q0 = d.ttd_q0;
  ga.x_ping_rows = x_rows;
  ga.x_guard = ttd ? d.ttd_guard : 0;
  ga.x_phase_rows = P * x_rows;
  ga.n_phase = d.n_phase;
  ga.tile_n = d.tile_n;
  ga.f16 = f16 ? 1 : 0;
  ga.nr = d.nr;
  ga.nr_x = d.nr_x;
  ga.n_beams = d.nb;
  ga.n_blank = d.n_blank;
  ga.r_min = (float)p->r_min_m;
  ga.dr = (float)d.dr;
  ga.alpha2 = (float)(2.0 * p->alpha_np_per_m);
  ga.gain = fp16 ? ctx->gain : nullptr;  // element echoes carry a gain only in the FP16 form
  ga.y_gain_inv = (float)(1.0 / (d.sep ? ctx->ysep_gain : ctx->y_gain));
  ga.env = o.env;
  ga.peak_keys = ctx->keys;
  ga.ping_max = ctx->pmax;
  ga.err = ctx->err_dev;
  CU(launch_gemm(ga, ctx->sm_count, st));
  mark(5);
  PeakArgs pa;
  pa.peak_keys = ctx->keys;
  pa.ping_max = ctx->pmax;
  pa.poses = ctx->poses;
  pa.n_pings = P;
  pa.n_beam_az = p->n_beam_az;
  pa.n_beam_el = p->n_beam_el;
  pa.nr = d.nr;
  pa.az0 = (float)(-p->hfov_rad / 2);
  pa.daz = (float)(p->hfov_rad / p->n_beam_az);
  pa.el0 = (float)(-p->vfov_rad / 2);
  pa.del = (float)(p->vfov_rad / p->n_beam_el);
  pa.r_min = (float)p->r_min_m;
  pa.dr = (float)d.dr;
  pa.thr_mode = p->thr_mode;
  pa.thr = (float)p->thr;
  pa.cloud = o.cloud;
  pa.cap = o.cap;
  pa.n_cloud = ctx->n_cloud_dev;
  pa.n_cloud_host = o.n_cloud_map;
  pa.counters_host = o.counters_map;
  pa.n_hits = ctx->n_hits;
  pa.err = ctx->err_dev;
  CU(launch_peaks(pa, st));
  mark(6);
  // results back to the host: staged outputs, per-ping point counts, hit count, error bits
  if (o.env_host)
    CU(cudaMemcpyAsync(o.env_host, o.env, sizeof(float) * o.env_elems, cudaMemcpyDeviceToHost, st));
  if (o.cloud_host && o.cap > 0)
    CU(cudaMemcpyAsync(o.cloud_host, o.cloud, sizeof(sonar_point) * P * o.cap, cudaMemcpyDeviceToHost, st));
  // (point counts, hit count and error bits reach the host through k_peaks' mapped writes)
  return SONAR_OK;
}

int check_call(sonar_ctx* ctx, const sonar_pose* poses, int P, const sonar_params* p, const sonar_ssp* ssp,
               const float* env, const sonar_point* cloud, int64_t cloud_cap) {
  if (!poses || P < 1) return fail(ctx, SONAR_E_ARG, "need at least one pose");
  if (!env) return fail(ctx, SONAR_E_ARG, "env is NULL");
  if (cloud_cap < 0 || (cloud_cap > 0 && !cloud)) return fail(ctx, SONAR_E_ARG, "bad cloud buffer");
  if (!ctx->has_scene) return fail(ctx, SONAR_E_NOSCENE, "no scene uploaded");
  int rc = validate(ctx, p, ssp);
  if (rc) return rc;
  for (int i = 0; i < P; ++i) {
    const double* q = poses[i].q;
    double n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(n2 > 1e-12) || !isfinite(poses[i].t[0] + poses[i].t[1] + poses[i].t[2]))
      return fail(ctx, SONAR_E_ARG, "pose %d is not finite or has a zero quaternion", i);
  }
  return SONAR_OK;
}

// Error bits and point counts of a finished call, as the caller sees them.
int report(sonar_ctx* ctx, int errw, const long long* n_cloud_host, int P, int64_t* n_cloud, int64_t cloud_cap,
           bool cloud_given) {
  if (errw & kErrTimeout) return fail(ctx, SONAR_E_TIMEOUT, "a device-side wait exceeded its limit");
  if (errw & kErrLoop) return fail(ctx, SONAR_E_TIMEOUT, "a ray-marching loop exceeded its step limit");
  if (errw & kErrStack) return fail(ctx, SONAR_E_TIMEOUT, "BVH traversal stack overflow");
  if (errw & kErrCapacity) return fail(ctx, SONAR_E_CAPACITY, "hit capacity %lld exceeded", (long long)ctx->hit_cap);
  int over = 0;
  for (int i = 0; i < P; ++i) {
    if (n_cloud) n_cloud[i] = n_cloud_host[i];
    if (n_cloud_host[i] > cloud_cap) over = 1;
  }
  if (over && cloud_given)
    return fail(ctx, SONAR_E_CAPACITY, "cloud needs more than %lld points per ping", (long long)cloud_cap);
  return SONAR_OK;
}

// Captured graphs bake in options and buffers: they are rebuilt after an option, the
// volume scatterers or the scene change.
void drop_graphs(sonar_ctx* ctx) {
  for (auto& e : ctx->graphs) cudaGraphExecDestroy(e.exec);
  ctx->graphs.clear();
  for (AsyncSlot& sl : ctx->aslot)
    if (sl.gexec) { cudaGraphExecDestroy(sl.gexec); sl.gexec = nullptr; sl.gkey.clear(); }
}

// Waits for an asynchronous slot's ping and hands its counts and errors back.
int retire(sonar_ctx* ctx, AsyncSlot& sl) {
  if (!sl.busy) return SONAR_OK;
  sl.busy = false;
  CU(cudaEventSynchronize(sl.ev_done));
  CU(cudaStreamWaitEvent(ctx->user_stream, sl.ev_done, 0));
  ctx->stats.n_hits = (int64_t)sl.counters_host[0];
  return report(ctx, (int)sl.counters_host[1], sl.n_cloud_host, sl.P, sl.n_cloud_user, sl.cloud_cap, sl.cloud_given);
}

// Retires every asynchronous ping in flight, oldest first; returns the first error.
int drain(sonar_ctx* ctx) {
  int first = SONAR_OK;
  for (int k = 0; k < 2; ++k) {
    const int rc = retire(ctx, ctx->aslot[(ctx->next_slot + k) & 1]);
    if (rc && first == SONAR_OK) first = rc;
  }
  return first;
}

// Everything a captured pipeline bakes in: shapes and parameters, output and host-word
// pointers, options, the scene version, the profile and the workspace buffers (a
// workspace regrow moves them). Options, volume scatterers, fields and scene uploads also
// drop every graph outright.
std::vector<uint8_t> pipeline_key(const sonar_ctx* ctx, int P, const sonar_params* p, const sonar_ssp* ssp,
                                  const Derived& d, const Outputs& o) {
  std::vector<uint8_t> k;
  key_add(k, P); key_add(k, *p); key_add(k, o.env); key_add(k, o.cloud); key_add(k, o.cap);
  key_add(k, o.env_host); key_add(k, o.cloud_host); key_add(k, o.pose_src); key_add(k, o.counters_map);
  key_add(k, o.n_cloud_map);
  key_add(k, ctx->debug); key_add(k, ctx->timing); key_add(k, ctx->synth_opt); key_add(k, ctx->scene_version);
  key_add(k, ctx->raw_u); key_add(k, ctx->ttd_u);
  key_add(k, d.c_ref);
  key_add(k, d.tile_n); key_add(k, ctx->cur_pairs); key_add(k, ctx->gemm_cluster);
  if (ssp) {
    key_add(k, ssp->n_nodes);
    for (int i = 0; i < ssp->n_nodes; ++i) { key_add(k, ssp->c[i]); if (ssp->z) key_add(k, ssp->z[i]); }
  }
  key_add(k, ctx->vol_order);
  key_add(k, ctx->hits); key_add(k, ctx->S); key_add(k, ctx->x_hi); key_add(k, ctx->y_hi); key_add(k, ctx->keys);
  key_add(k, d.sep); key_add(k, ctx->ysep_hi); key_add(k, ctx->sep_fz); key_add(k, ctx->rank);
  return k;
}

// ------------------------------------------------------------------ autotuner
// The choices the tuner owns are those the caller left to the library (SONAR_OPT_TILE_N
// and SONAR_OPT_SYNTH at 0); they are keyed by what changes the best tile: the ping
// count, the range and beam grids, the array, the precision, the raw phases, the pulse
// and range extent (taps per hit) and the beamforming option (separable or dense).
std::vector<uint8_t> tune_key(const sonar_ctx* ctx, int P, const sonar_params* p) {
  std::vector<uint8_t> k;
  key_add(k, P); key_add(k, p->n_range); key_add(k, p->n_beam_az); key_add(k, p->n_beam_el);
  key_add(k, p->nx); key_add(k, p->ny); key_add(k, p->precision); key_add(k, ctx->raw_u); key_add(k, ctx->ttd_u);
  key_add(k, p->pulse_s); key_add(k, p->r_max_m - p->r_min_m); key_add(k, ctx->tile_opt); key_add(k, ctx->synth_opt);
  key_add(k, ctx->bf_opt);
  return k;
}

// Sets the current call's tile choices from the cache; false when the key was not tuned.
bool tune_lookup(sonar_ctx* ctx, const std::vector<uint8_t>& key) {
  ctx->cur_tile_n = 0;
  ctx->cur_pairs = 0;
  ctx->cur_tuned = false;
  if (!ctx->autotune) return true;
  for (const auto& e : ctx->tuned)
    if (e.key == key) {
      ctx->cur_tile_n = e.tile_n;
      ctx->cur_pairs = e.pairs;
      ctx->cur_tuned = true;
      return true;
    }
  return false;
}

// Times the pipeline eagerly with per-stage events, min of three after one warm-up:
// the beamforming GEMM at each N tile, then the synthesis at each tile width (with the
// best N), and keeps the fastest of each. The runs compute the call's own pings into
// its own outputs, so they leave valid results behind.
int autotune(sonar_ctx* ctx, int P, const sonar_params* p, const sonar_ssp* ssp, double xs, double zs,
             const Outputs& o, const std::vector<uint8_t>& key) {
  const bool saved_timing = ctx->timing;
  ctx->timing = true;
  int rc = SONAR_OK;
  auto measure = [&](float* ms_synth, float* ms_gemm) -> int {
    Derived d;
    int r;
    if ((r = derive(ctx, p, ssp, xs, zs, P, d))) return r;
    if ((r = ensure_tables(ctx, p, d))) return r;
    if ((r = ensure_workspace(ctx, P, d))) return r;
    float bs = 1e30f, bg = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      int kernels = 0;
      if ((r = enqueue(ctx, P, p, d, o, &kernels))) return r;
      CU(cudaStreamSynchronize(ctx->stream));
      if (rep == 0) continue;
      float ts = 0.f, tg = 0.f;
      CU(cudaEventElapsedTime(&ts, ctx->stage_ev[2], ctx->stage_ev[3]));
      CU(cudaEventElapsedTime(&tg, ctx->stage_ev[4], ctx->stage_ev[5]));
      bs = fminf(bs, ts);
      bg = fminf(bg, tg);
    }
    *ms_synth = bs;
    *ms_gemm = bg;
    return SONAR_OK;
  };
  sonar_ctx::TuneEntry e;
  e.key = key;
  float best_g = 1e30f, best_s = 1e30f, ms_s = 0.f, ms_g = 0.f;
  int best_n = 0, best_p = 0;
  if (ctx->tile_opt == 0) {
    for (int bn : {256, 224, 192, 128}) {
      // separable beams take only N tiles inside one elevation row (derive() would
      // replace the others and time the same tile twice)
      Derived dt;
      ctx->cur_tile_n = 0;
      if (derive(ctx, p, ssp, xs, zs, P, dt) == SONAR_OK && dt.sep && p->n_beam_az % (bn / 2) != 0) continue;
      ctx->cur_tile_n = bn;
      if ((rc = measure(&ms_s, &ms_g))) break;
      if (ms_g < best_g) { best_g = ms_g; best_n = bn; }
    }
  }
  ctx->cur_tile_n = best_n;
  Derived d0;
  if (!rc && (rc = derive(ctx, p, ssp, xs, zs, P, d0)) == SONAR_OK && ctx->synth_opt == 0 &&
      synth_tz_applies(p->nx, p->ny, d0.taps)) {
    for (int np : {96, 64, 32}) {
      ctx->cur_pairs = np;
      if ((rc = measure(&ms_s, &ms_g))) break;
      if (ms_s < best_s) { best_s = ms_s; best_p = np; }
    }
  }
  ctx->timing = saved_timing;
  if (rc) {
    ctx->cur_tile_n = ctx->cur_pairs = 0;
    return rc;
  }
  e.tile_n = best_n;
  e.pairs = best_p;
  e.ms_gemm = best_g;
  e.ms_synth = best_s;
  ctx->tuned.push_back(e);
  ctx->cur_tile_n = best_n;
  ctx->cur_pairs = best_p;
  ctx->cur_tuned = true;
  return SONAR_OK;
}

int run(sonar_ctx* ctx, const sonar_pose* poses, int P, const sonar_params* p, const sonar_ssp* ssp, float* env,
        sonar_point* cloud, int64_t cloud_cap, int64_t* n_cloud) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  int rc = check_call(ctx, poses, P, p, ssp, env, cloud, cloud_cap);
  if (rc) return rc;
  CU(cudaSetDevice(ctx->device));
  // asynchronous pings still in flight finish first (and report their errors here)
  if ((rc = drain(ctx))) return rc;
  // the work stream starts after everything already queued on the caller's stream
  CU(cudaEventRecord(ctx->ev_in, ctx->user_stream));
  CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
  const std::vector<uint8_t> tkey = tune_key(ctx, P, p);
  const bool tuned = tune_lookup(ctx, tkey);
  Derived d;
  if ((rc = derive(ctx, p, ssp, poses[0].t[0], poses[0].t[2], P, d))) return rc;
  if ((int64_t)P * d.nr_pad + 1 > (1LL << 31) - 1) return fail(ctx, SONAR_E_UNSUPPORTED, "batch too large");
  if ((rc = ensure_tables(ctx, p, d))) return rc;
  if ((rc = ensure_workspace(ctx, P, d))) return rc;

  // outputs: device buffers and mapped pinned host buffers are written in place, other
  // host buffers through staging
  void* env_d = nullptr;
  void* cloud_d = nullptr;
  const bool env_dev = classify(env, &env_d) != Mem::Host;
  const bool cloud_dev = cloud_cap == 0 || classify(cloud, &cloud_d) != Mem::Host;
  const int64_t env_elems = (int64_t)P * d.nb * d.nr;
  Outputs o;
  o.env = static_cast<float*>(env_d);
  o.env_host = nullptr;
  o.env_elems = env_elems;
  if (!env_dev) {
    if ((rc = grow(ctx, ctx->env_stage, ctx->env_cap, env_elems, sizeof(float), false))) return rc;
    o.env = ctx->env_stage;
    o.env_host = env;
  }
  o.cap = cloud_cap;
  o.cloud = cloud_cap == 0 ? cloud : static_cast<sonar_point*>(cloud_d);
  o.cloud_host = nullptr;
  if (!cloud_dev) {
    if ((rc = grow(ctx, ctx->cloud_stage, ctx->cloud_stage_cap, (int64_t)P * cloud_cap, sizeof(sonar_point), false)))
      return rc;
    o.cloud = ctx->cloud_stage;
    o.cloud_host = cloud;
  }
  if (!ctx->counters_host) {
    CU(cudaMallocHost(&ctx->counters_host, 3 * sizeof(unsigned long long)));
    CU(cudaHostGetDevicePointer((void**)&ctx->counters_map, ctx->counters_host, 0));
  }
  ctx->counters_host[1] = 0;
  o.pose_src = ctx->pose_map;
  o.n_cloud_map = ctx->n_cloud_map;
  o.counters_map = ctx->counters_map;

  // the graph's first node copies these to the device
  for (int i = 0; i < P; ++i) ctx->pose_host[i] = dev_pose(poses[i]);

  // first call of this shape: the autotuner times the candidate tiles, then the call
  // proceeds with the winners
  if (!tuned) {
    if ((rc = autotune(ctx, P, p, ssp, poses[0].t[0], poses[0].t[2], o, tkey))) return rc;
    if ((rc = derive(ctx, p, ssp, poses[0].t[0], poses[0].t[2], P, d))) return rc;
    if ((rc = ensure_tables(ctx, p, d))) return rc;
    if ((rc = ensure_workspace(ctx, P, d))) return rc;
  }

  const bool timed = ctx->timing;
  int kernels = 0;
  // stage events cannot be timed when recorded by graph nodes: timing runs eagerly
  if (ctx->use_graph && !timed) {
    const std::vector<uint8_t> k = pipeline_key(ctx, P, p, ssp, d, o);
    sonar_ctx::GraphEntry* ge = nullptr;
    for (auto& e : ctx->graphs)
      if (e.key == k) ge = &e;
    if (!ge) {
      constexpr size_t kMaxGraphs = 4;
      if (ctx->graphs.size() == kMaxGraphs) {  // evict the least recently used
        auto lru = ctx->graphs.begin();
        for (auto it = ctx->graphs.begin(); it != ctx->graphs.end(); ++it)
          if (it->used < lru->used) lru = it;
        cudaGraphExecDestroy(lru->exec);
        ctx->graphs.erase(lru);
      }
      sonar_ctx::GraphEntry e;
      cudaGraph_t g;
      CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      rc = enqueue(ctx, P, p, d, o, &e.kernels);
      cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
      if (rc) { if (ce == cudaSuccess) cudaGraphDestroy(g); return rc; }
      CU(ce);
      cudaError_t ie = cudaGraphInstantiate(&e.exec, g, 0);
      cudaGraphDestroy(g);
      CU(ie);
      e.key = k;
      ctx->graphs.push_back(std::move(e));
      ge = &ctx->graphs.back();
    }
    ge->used = ++ctx->graph_tick;
    CU(cudaGraphLaunch(ge->exec, ctx->stream));
    kernels = ge->kernels;
  } else {
    rc = enqueue(ctx, P, p, d, o, &kernels);
  }
  if (rc) return rc;
  CU(cudaEventRecord(ctx->ev_out, ctx->stream));
  CU(cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0));
  CU(cudaStreamSynchronize(ctx->stream));
  const unsigned long long nh = ctx->counters_host[0];
  const int errw = (int)ctx->counters_host[1];
  ctx->last_p = P;
  ctx->last_d = d;
  ctx->last_raw_u = ctx->raw_u > 0 ? ctx->raw_u : ctx->ttd_u;
  ctx->last_ttd_u = ctx->ttd_u;
  ctx->last_params = *p;
  ctx->stats.n_hits = (int64_t)nh;
  ctx->stats.hit_capacity = ctx->hit_cap;
  ctx->stats.n_pings = P;
  ctx->stats.taps = d.taps;
  ctx->stats.kernels = kernels;
  ctx->stats.synth_mma_flop = (double)ctx->counters_host[2];
  ctx->stats.tile_n = d.tile_n;
  static const int32_t kCols[5] = {0, 0, 32, 64, 96};
  ctx->stats.synth_cols = ctx->synth_opt >= 2 ? kCols[ctx->synth_opt] : ctx->cur_pairs;
  ctx->stats.autotuned = ctx->cur_tuned ? 1 : 0;
  ctx->stats.gemm_cluster = gemm_cluster_for(ctx, P * d.nr_x / 128, d);
  ctx->stats.beam_sep = d.sep;
  if (timed) {
    float t[6];
    for (int i = 0; i < 6; ++i) CU(cudaEventElapsedTime(&t[i], ctx->stage_ev[i], ctx->stage_ev[i + 1]));
    ctx->stats.ms_trace = t[0];
    ctx->stats.ms_bin = t[1];
    ctx->stats.ms_synth = t[2];
    ctx->stats.ms_convert = t[3];
    ctx->stats.ms_beamform = t[4];
    ctx->stats.ms_peaks = t[5];
  }
  return report(ctx, errw, ctx->n_cloud_host, P, n_cloud, cloud_cap, cloud_cap > 0 || cloud);
}

// Asynchronous pings (sonar_ping_async): the pipeline of `run` on one of two slots. The
// slot's previous ping (two submissions back) is retired first, so at most two pings
// are in flight. An envelope bound for pinned host memory is written to the slot's
// device staging and copied by a copy engine on the copy stream, overlapping the next
// ping's ray casting and synthesis instead of slowing the GEMM epilogue with writes
// across the host link.
int run_async(sonar_ctx* ctx, const sonar_pose* poses, int P, const sonar_params* p, const sonar_ssp* ssp,
              float* env, sonar_point* cloud, int64_t cloud_cap, int64_t* n_cloud) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  int rc = check_call(ctx, poses, P, p, ssp, env, cloud, cloud_cap);
  if (rc) return rc;
  CU(cudaSetDevice(ctx->device));
  void* env_d = nullptr;
  void* cloud_d = nullptr;
  const Mem env_kind = classify(env, &env_d);
  const Mem cloud_kind = cloud_cap == 0 ? Mem::Device : classify(cloud, &cloud_d);
  if (env_kind == Mem::Host || cloud_kind == Mem::Host)
    return fail(ctx, SONAR_E_ARG, "asynchronous pings need device or pinned host outputs");
  // first call of this shape: tuned by one synchronous call (into these outputs)
  if (!tune_lookup(ctx, tune_key(ctx, P, p))) {
    if ((rc = run(ctx, poses, P, p, ssp, env, cloud, cloud_cap, nullptr))) return rc;
    if (!tune_lookup(ctx, tune_key(ctx, P, p))) return fail(ctx, SONAR_E_CUDA, "autotuner left no entry");
  }
  const int s = ctx->next_slot;
  AsyncSlot& sl = ctx->aslot[s];
  const int rc_prev = retire(ctx, sl);
  ctx->next_slot ^= 1;
  CU(cudaEventRecord(ctx->ev_in, ctx->user_stream));
  CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
  Derived d;
  if ((rc = derive(ctx, p, ssp, poses[0].t[0], poses[0].t[2], P, d))) return rc;
  if ((int64_t)P * d.nr_pad + 1 > (1LL << 31) - 1) return fail(ctx, SONAR_E_UNSUPPORTED, "batch too large");
  if ((rc = ensure_tables(ctx, p, d))) return rc;
  if ((rc = ensure_workspace(ctx, P, d))) return rc;
  if (P > sl.p_cap) {
    if (sl.pose_host) cudaFreeHost(sl.pose_host);
    if (sl.n_cloud_host) cudaFreeHost(sl.n_cloud_host);
    sl.pose_host = nullptr;
    sl.n_cloud_host = nullptr;
    sl.p_cap = 0;
    CU(cudaMallocHost(&sl.pose_host, sizeof(DevPose) * P));
    CU(cudaHostGetDevicePointer((void**)&sl.pose_map, sl.pose_host, 0));
    CU(cudaMallocHost(&sl.n_cloud_host, sizeof(long long) * P));
    CU(cudaHostGetDevicePointer((void**)&sl.n_cloud_map, sl.n_cloud_host, 0));
    sl.p_cap = P;
  }
  if (!sl.counters_host) {
    CU(cudaMallocHost(&sl.counters_host, 3 * sizeof(unsigned long long)));
    CU(cudaHostGetDevicePointer((void**)&sl.counters_map, sl.counters_host, 0));
  }
  if (!sl.ev_done) {
    CU(cudaEventCreateWithFlags(&sl.ev_done, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&sl.ev_gemm, cudaEventDisableTiming));
  }
  if (!ctx->copy_stream) CU(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  const int64_t env_elems = (int64_t)P * d.nb * d.nr;
  const bool staged = env_kind == Mem::Mapped;
  Outputs o;
  o.env = static_cast<float*>(env_d);
  if (staged) {
    if ((rc = grow(ctx, sl.env_stage, sl.env_cap, env_elems, sizeof(float), false))) return rc;
    o.env = sl.env_stage;
  }
  o.env_host = nullptr;
  o.env_elems = env_elems;
  o.cap = cloud_cap;
  o.cloud = cloud_cap == 0 ? cloud : static_cast<sonar_point*>(cloud_d);
  o.cloud_host = nullptr;
  o.pose_src = sl.pose_map;
  o.n_cloud_map = sl.n_cloud_map;
  o.counters_map = sl.counters_map;
  sl.counters_host[0] = 0;
  sl.counters_host[1] = 0;
  for (int i = 0; i < P; ++i) sl.pose_host[i] = dev_pose(poses[i]);

  int kernels = 0;
  if (ctx->use_graph && !ctx->timing) {
    const std::vector<uint8_t> k = pipeline_key(ctx, P, p, ssp, d, o);
    if (!sl.gexec || k != sl.gkey) {
      if (sl.gexec) { cudaGraphExecDestroy(sl.gexec); sl.gexec = nullptr; }
      cudaGraph_t g;
      CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      rc = enqueue(ctx, P, p, d, o, &sl.graph_kernels);
      cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
      if (rc) { if (ce == cudaSuccess) cudaGraphDestroy(g); return rc; }
      CU(ce);
      cudaError_t ie = cudaGraphInstantiate(&sl.gexec, g, 0);
      cudaGraphDestroy(g);
      CU(ie);
      sl.gkey = k;
    }
    CU(cudaGraphLaunch(sl.gexec, ctx->stream));
    kernels = sl.graph_kernels;
  } else {
    if ((rc = enqueue(ctx, P, p, d, o, &kernels))) return rc;
  }
  if (staged) {
    CU(cudaEventRecord(sl.ev_gemm, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->copy_stream, sl.ev_gemm, 0));
    CU(cudaMemcpyAsync(env, sl.env_stage, sizeof(float) * env_elems, cudaMemcpyDeviceToHost, ctx->copy_stream));
    CU(cudaEventRecord(sl.ev_done, ctx->copy_stream));
  } else {
    CU(cudaEventRecord(sl.ev_done, ctx->stream));
  }
  // (the caller's stream is ordered after this call's outputs when the call is retired:
  // ordering it now would chain the next call's work behind this call's envelope copy)
  sl.busy = true;
  sl.P = P;
  sl.n_cloud_user = n_cloud;
  sl.cloud_cap = cloud_cap;
  sl.cloud_given = cloud_cap > 0 || cloud;
  ctx->last_p = P;
  ctx->last_d = d;
  ctx->last_raw_u = ctx->raw_u > 0 ? ctx->raw_u : ctx->ttd_u;
  ctx->last_ttd_u = ctx->ttd_u;
  ctx->last_params = *p;
  ctx->stats.hit_capacity = ctx->hit_cap;
  ctx->stats.n_pings = P;
  ctx->stats.taps = d.taps;
  ctx->stats.kernels = kernels;
  return rc_prev;
}


// ------------------------------------------------------------------ learned surrogate
constexpr int kSurBufs = 7;          // a1..a5 and two back-propagated gradients
constexpr int64_t kSurChunk = 8192;  // beams per inference pass

int sur_alloc_params(sonar_ctx* ctx) {
  auto& S = ctx->sur;
  if (S.params) return SONAR_OK;
  CU(cudaMalloc(&S.params, sizeof(float) * 4 * kSurParams));
  CU(cudaMemset(S.params, 0, sizeof(float) * 4 * kSurParams));
  const int64_t wn = 4LL * kSurK * kSurC * kSurC;
  CU(cudaMalloc(&S.wbf, sizeof(__nv_bfloat16) * 2 * wn));
  CU(cudaMalloc(&S.wsmall, sizeof(float) * (kSurC * 4 * kSurK + kSurC * kSurK)));
  CU(cudaMalloc(&S.loss, sizeof(double)));
  S.net.theta = S.params;
  S.net.m = S.params + kSurParams;
  S.net.v = S.params + 2 * kSurParams;
  S.net.grad = S.params + 3 * kSurParams;
  S.net.wf = S.wbf;
  S.net.wb = S.wbf + wn;
  S.net.w_in = S.wsmall;
  S.net.w_out = S.wsmall + kSurC * 4 * kSurK;
  return SONAR_OK;
}

// Common checks and set-up of a surrogate call over P pings: parameters, the scene, the
// isovelocity restriction, the range grid, the poses on the device and the rendering
// of every beam of every ping into sur.feat.
int sur_begin(sonar_ctx* ctx, const sonar_pose* poses, int P, const sonar_params* p, const sonar_ssp* ssp,
              Derived& d) {
  int rc;
  if (!ctx->has_scene) return fail(ctx, SONAR_E_NOSCENE, "no scene uploaded");
  if (!poses || P < 1) return fail(ctx, SONAR_E_ARG, "need at least one pose");
  if ((rc = validate(ctx, p, ssp))) return rc;
  for (int i = 0; i < P; ++i) {
    const double* q = poses[i].q;
    double n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(n2 > 1e-12) || !isfinite(poses[i].t[0] + poses[i].t[1] + poses[i].t[2]))
      return fail(ctx, SONAR_E_ARG, "pose %d is not finite or has a zero quaternion", i);
  }
  if (!ctx->sur.has_weights) return fail(ctx, SONAR_E_ARG, "the surrogate has no weights (sonar_sur_set_weights)");
  CU(cudaSetDevice(ctx->device));
  if ((rc = drain(ctx))) return rc;
  if ((rc = derive(ctx, p, ssp, poses[0].t[0], poses[0].t[2], P, d))) return rc;
  if (d.curved || ctx->fld.nx > 0)
    return fail(ctx, SONAR_E_UNSUPPORTED, "the surrogate renders isovelocity routes only");
  if (d.nr % 256 != 0) return fail(ctx, SONAR_E_UNSUPPORTED, "the surrogate needs n_range a multiple of 256");
  auto& S = ctx->sur;
  if ((rc = grow(ctx, S.poses, S.poses_cap, P, sizeof(DevPose), false))) return rc;
  std::vector<DevPose> hp(P);
  for (int i = 0; i < P; ++i) hp[i] = dev_pose(poses[i]);
  CU(cudaEventRecord(ctx->ev_in, ctx->user_stream));
  CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
  CU(cudaMemcpyAsync(S.poses, hp.data(), sizeof(DevPose) * P, cudaMemcpyHostToDevice, ctx->stream));
  if ((rc = grow(ctx, S.feat, S.feat_cap, (int64_t)P * d.nb * 8, sizeof(float), false))) return rc;
  if (!ctx->err_dev) CU(cudaMalloc(&ctx->err_dev, sizeof(int)));
  CU(cudaMemsetAsync(ctx->err_dev, 0, sizeof(int), ctx->stream));
  TraceArgs ta = trace_args(ctx, P, p, d, false);
  ta.poses = S.poses;
  CU(launch_render(ta, p->n_beam_az, p->n_beam_el, p->hfov_rad, p->vfov_rad, S.feat, ctx->stream));
  return SONAR_OK;
}

// Activation and gradient buffers for `beams` beams of rb rows (zero padding rows
// included; they are zeroed here once and never written afterwards).
int sur_buffers(sonar_ctx* ctx, int64_t beams, int rb) {
  auto& S = ctx->sur;
  if (S.buf && beams <= S.beams_cap && rb == S.rb) return SONAR_OK;
  dfree(S.buf);
  S.beams_cap = 0;
  const int64_t rows = beams * rb;
  CU(cudaMalloc(&S.buf, sizeof(__nv_bfloat16) * kSurC * rows * kSurBufs));
  CU(cudaMemsetAsync(S.buf, 0, sizeof(__nv_bfloat16) * kSurC * rows * kSurBufs, ctx->stream));
  S.beams_cap = beams;
  S.rb = rb;
  return SONAR_OK;
}

__nv_bfloat16* sur_buf(sonar_ctx* ctx, int i) {
  return ctx->sur.buf + (int64_t)i * ctx->sur.beams_cap * ctx->sur.rb * kSurC;
}

// Forward pass of n_sel beams (rendering rows `beams`, or the n_feat rows of feat in
// order): layer 0, the four hidden layers on the tensor cores, the output layer.
// Training (target != null) leaves the loss gradient in sur.g; inference writes env.
int sur_forward(sonar_ctx* ctx, const float* feat, const int32_t* beams, int64_t n_sel, int64_t n_feat,
                const sonar_params* p, const Derived& d, const float* target, float* env) {
  auto& S = ctx->sur;
  int rc;
  const int rb = d.nr + 2 * kSurHalo;
  cudaStream_t st = ctx->stream;
  const double inv_dr = 1.0 / d.dr;
  CU(sur_input(feat, beams, n_sel, n_feat, d.nr, p->r_min_m, inv_dr, S.net, sur_buf(ctx, 0), rb, ctx->err_dev, st));
  for (int L = 1; L <= 4; ++L) {
    SurConvArgs ca;
    memset(&ca, 0, sizeof(ca));
    if ((rc = make_map(ctx, &ca.map_x, sur_buf(ctx, L - 1), n_sel * rb, kSurC, 128 + kSurK - 1, false))) return rc;
    if ((rc = make_map(ctx, &ca.map_w, S.net.wf + (int64_t)(L - 1) * kSurK * kSurC * kSurC, kSurK * kSurC, kSurC,
                       kSurC, false)))
      return rc;
    ca.bias = S.net.theta + sur_boff(L);
    ca.out = sur_buf(ctx, L);
    ca.n_tiles = n_sel * (d.nr / 128);
    ca.tiles_per_beam = d.nr / 128;
    ca.rb = rb;
    ca.err = ctx->err_dev;
    CU(sur_conv(ca, false, ctx->sm_count, st));
  }
  const float inv_scale = (float)(1.0 / S.e_scale);
  const float g_scale = (float)(2.0 / ((double)n_sel * d.nr));
  CU(sur_head(sur_buf(ctx, 4), S.net, n_sel, d.nr, rb, target, beams, n_feat, inv_scale, g_scale, S.g, S.loss, env,
              (float)S.e_scale, ctx->err_dev, st));
  return SONAR_OK;
}

// Backward pass after a training forward pass: gradients of every parameter into sur.grad.
int sur_backward(sonar_ctx* ctx, const float* feat, const int32_t* beams, int64_t n_sel, int64_t n_feat,
                 const sonar_params* p, const Derived& d) {
  auto& S = ctx->sur;
  int rc;
  const int rb = d.nr + 2 * kSurHalo;
  cudaStream_t st = ctx->stream;
  CU(sur_head_bwd(sur_buf(ctx, 4), S.g, S.net, n_sel, d.nr, rb, sur_buf(ctx, 5), st));
  int dz = 5;  // buffer of dz_{L+1}
  for (int L = 4; L >= 1; --L) {
    SurDwArgs wa;
    memset(&wa, 0, sizeof(wa));
    if ((rc = make_map(ctx, &wa.map_x, sur_buf(ctx, L - 1), n_sel * rb, kSurC, 80, false))) return rc;
    if ((rc = make_map(ctx, &wa.map_dz, sur_buf(ctx, dz), n_sel * rb, kSurC, 80, false))) return rc;
    wa.grad_w = S.net.grad + sur_woff(L);
    wa.grad_b = S.net.grad + sur_boff(L);
    wa.kb_per_beam = d.nr / 64 + 1;
    wa.n_kb = n_sel * wa.kb_per_beam;
    wa.nr = d.nr;
    wa.rb = rb;
    wa.err = ctx->err_dev;
    CU(sur_dw(wa, ctx->sm_count, st));
    SurConvArgs ca;
    memset(&ca, 0, sizeof(ca));
    if ((rc = make_map(ctx, &ca.map_x, sur_buf(ctx, dz), n_sel * rb, kSurC, 128 + kSurK - 1, false))) return rc;
    if ((rc = make_map(ctx, &ca.map_w, S.net.wb + (int64_t)(L - 1) * kSurK * kSurC * kSurC, kSurK * kSurC, kSurC,
                       kSurC, false)))
      return rc;
    ca.mask = sur_buf(ctx, L - 1);
    ca.out = sur_buf(ctx, 11 - dz);  // the other gradient buffer
    ca.n_tiles = n_sel * (d.nr / 128);
    ca.tiles_per_beam = d.nr / 128;
    ca.rb = rb;
    ca.err = ctx->err_dev;
    CU(sur_conv(ca, true, ctx->sm_count, st));
    dz = 11 - dz;
  }
  CU(sur_l1_dw(feat, beams, n_sel, n_feat, d.nr, p->r_min_m, 1.0 / d.dr, sur_buf(ctx, dz), rb, S.net, st));
  return SONAR_OK;
}

// Waits for the work stream, orders the caller's stream after it and turns the device
// error word into a return code.
int sur_finish(sonar_ctx* ctx) {
  CU(cudaEventRecord(ctx->ev_out, ctx->stream));
  CU(cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0));
  CU(cudaStreamSynchronize(ctx->stream));
  int errw = 0;
  CU(cudaMemcpy(&errw, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (errw & kErrIndex) return fail(ctx, SONAR_E_ARG, "a beam index lies outside the rendered beams");
  if (errw & kErrTimeout) return fail(ctx, SONAR_E_TIMEOUT, "a device-side wait exceeded its limit");
  if (errw & (kErrLoop | kErrStack)) return fail(ctx, SONAR_E_TIMEOUT, "ray casting exceeded a loop or stack limit");
  return SONAR_OK;
}

}  // namespace

extern "C" {

int sonar_create(sonar_ctx** out, int device, void* cuda_stream) {
  if (!out) return SONAR_E_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return SONAR_E_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return SONAR_E_CUDA;
  if (!(prop.major == 10 && prop.minor == 3)) return SONAR_E_UNSUPPORTED;
  if (cudaSetDevice(device) != cudaSuccess) return SONAR_E_CUDA;
  if (prepare_gemm() != cudaSuccess || prepare_synth_tc() != cudaSuccess || sur_conv_prepare() != cudaSuccess ||
      prepare_synth_wb() != cudaSuccess)
    return SONAR_E_CUDA;
  sonar_ctx* c = new (std::nothrow) sonar_ctx();
  if (!c) return SONAR_E_NOMEM;
  c->device = device;
  c->user_stream = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    delete c;
    return SONAR_E_CUDA;
  }
  for (auto& e : c->stage_ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
    delete c;
    return SONAR_E_CUDA;
  }
  c->sm_count = prop.multiProcessorCount;
  *out = c;
  return SONAR_OK;
}

int sonar_set_stream(sonar_ctx* ctx, void* cuda_stream) {
  if (!ctx) return SONAR_E_ARG;
  ctx->user_stream = (cudaStream_t)cuda_stream;
  return SONAR_OK;
}

const char* sonar_last_error(const sonar_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int sonar_set_option(sonar_ctx* ctx, int32_t option, int64_t value) {
  if (!ctx) return SONAR_E_ARG;
  switch (option) {
    case SONAR_OPT_DEBUG: ctx->debug = value != 0; break;
    case SONAR_OPT_TIMING: ctx->timing = value != 0; break;
    case SONAR_OPT_GRAPH: ctx->use_graph = value != 0; break;
    case SONAR_OPT_SYNTH:
      if (value < 0 || value > 4) return fail(ctx, SONAR_E_ARG, "synthesis option must be 0 to 4");
      ctx->synth_opt = (int)value;
      break;
    case SONAR_OPT_RAW:
      if (value < 0 || value > 8) return fail(ctx, SONAR_E_ARG, "raw series: 0 (off) or 1 to 8 samples per cell");
      ctx->raw_u = (int)value;
      break;
    case SONAR_OPT_GEMM_CLUSTER:
      if (value != 0 && value != 1 && value != 2 && value != 4)
        return fail(ctx, SONAR_E_ARG, "beamforming cluster: 0 (automatic), 1, 2 or 4");
      ctx->gemm_cluster = (int)value;
      break;
    case SONAR_OPT_TTD:
      if (value < 0 || value > 8) return fail(ctx, SONAR_E_ARG, "true-time delay: 0 (off) or 1 to 8 phases per cell");
      ctx->ttd_u = (int)value;
      break;
    case SONAR_OPT_BVH:
      if (value != 0 && value != 1) return fail(ctx, SONAR_E_ARG, "BVH build: 0 (SAH) or 1 (Morton order)");
      ctx->bvh_opt = (int)value;
      break;
    case SONAR_OPT_TRAVERSAL:
      if (value != 0 && value != 1) return fail(ctx, SONAR_E_ARG, "traversal: 0 (per thread) or 1 (per warp)");
      ctx->traversal = (int)value;
      drop_graphs(ctx);
      break;
    case SONAR_OPT_AUTOTUNE:
      if (value != 0 && value != 1) return fail(ctx, SONAR_E_ARG, "autotune: 0 (off) or 1 (on)");
      ctx->autotune = (int)value;
      break;
    case SONAR_OPT_CROSS:
      if (value != 0 && value != 1) return fail(ctx, SONAR_E_ARG, "cross terms: 0 (off) or 1 (on)");
      ctx->cross = (int)value;
      break;
    case SONAR_OPT_BEAMFORM:
      if (value != 0 && value != 1) return fail(ctx, SONAR_E_ARG, "beamforming: 0 (separable where it applies) or 1 (dense)");
      ctx->bf_opt = (int)value;
      break;
    case SONAR_OPT_TILE_N:
      if (value != 0 && value != 128 && value != 192 && value != 224 && value != 256)
        return fail(ctx, SONAR_E_ARG, "tile_n must be 0, 128, 192, 224 or 256");
      ctx->tile_opt = (int)value;
      break;
    default: return fail(ctx, SONAR_E_ARG, "unknown option %d", option);
  }
  drop_graphs(ctx);
  return SONAR_OK;
}

int sonar_set_field(sonar_ctx* ctx, const sonar_field* f) {
  if (!ctx) return SONAR_E_ARG;
  CU(cudaSetDevice(ctx->device));
  {
    const int rc = drain(ctx);
    if (rc) return rc;
  }
  if (!f || f->nx == 0) {
    ctx->fld = sonar_field{};
  } else {
    if (f->nx < 2 || f->nz < 2 || !(f->dx > 0) || !(f->dz > 0) || !(f->step_m > 0) || !f->c ||
        !isfinite(f->x0) || !isfinite(f->z0))
      return fail(ctx, SONAR_E_ARG, "field: nx, nz >= 2, dx, dz, step > 0 and a grid are required");
    const int64_t n = (int64_t)f->nx * f->nz;
    for (int64_t k = 0; k < n; ++k)
      if (!(f->c[k] > 0) || !isfinite(f->c[k])) return fail(ctx, SONAR_E_ARG, "field speeds must be positive");
    CU(cudaStreamSynchronize(ctx->stream));
    dfree(ctx->fld_c);
    CU(cudaMalloc(&ctx->fld_c, sizeof(double) * n));
    CU(cudaMemcpy(ctx->fld_c, f->c, sizeof(double) * n, cudaMemcpyHostToDevice));
    ctx->fld_host.assign(f->c, f->c + n);
    ctx->fld = *f;
    ctx->fld.c = ctx->fld_host.data();
  }
  drop_graphs(ctx);
  return SONAR_OK;
}

int sonar_set_volume(sonar_ctx* ctx, const sonar_volume* v) {
  if (!ctx) return SONAR_E_ARG;
  if (!v || v->n == 0) {
    ctx->vol_n = 0;
  } else {
    if (v->n < 0 || v->n > (1LL << 28)) return fail(ctx, SONAR_E_ARG, "volume scatterers: 0 to 2^28");
    double V = 1.0;
    for (int k = 0; k < 3; ++k) {
      if (!(v->hi[k] > v->lo[k])) return fail(ctx, SONAR_E_ARG, "volume box must have hi > lo on every axis");
      V *= v->hi[k] - v->lo[k];
    }
    if (!(v->s_v >= 0)) return fail(ctx, SONAR_E_ARG, "volume backscattering coefficient must be >= 0");
    ctx->vol_n = v->n;
    for (int k = 0; k < 3; ++k) { ctx->vol_lo[k] = v->lo[k]; ctx->vol_hi[k] = v->hi[k]; }
    ctx->vol_sigma = sqrt(v->s_v * V / (double)v->n);
  }
  drop_graphs(ctx);
  return SONAR_OK;
}

static void free_scene(sonar_ctx* c) {
  dfree(c->tri32); dfree(c->triv); dfree(c->tri_prim); dfree(c->tri_mu); dfree(c->tri_flags);
  dfree(c->tri_plane); dfree(c->tri_inv_n);
  dfree(c->nodes); dfree(c->points); dfree(c->planes);
  c->has_scene = false;
  memset(&c->sc, 0, sizeof(c->sc));
}

int sonar_destroy(sonar_ctx* c) {
  if (!c) return SONAR_OK;
  cudaSetDevice(c->device);
  drain(c);
  cudaStreamSynchronize(c->stream);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  drop_graphs(c);
  for (AsyncSlot& sl : c->aslot) {
    if (sl.pose_host) cudaFreeHost(sl.pose_host);
    if (sl.n_cloud_host) cudaFreeHost(sl.n_cloud_host);
    if (sl.counters_host) cudaFreeHost(sl.counters_host);
    if (sl.ev_done) cudaEventDestroy(sl.ev_done);
    if (sl.ev_gemm) cudaEventDestroy(sl.ev_gemm);
    dfree(sl.env_stage);
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  for (auto& e : c->stage_ev)
    if (e) cudaEventDestroy(e);
  if (c->stream) cudaStreamDestroy(c->stream);
  free_scene(c);
  dfree(c->ray_dirs); dfree(c->ray_dirs32); dfree(c->row_domega); dfree(c->y_hi); dfree(c->y_lo); dfree(c->rtab); dfree(c->taper_dev);
  dfree(c->beam_uyz);
  if (c->pose_host) cudaFreeHost(c->pose_host);
  if (c->n_cloud_host) cudaFreeHost(c->n_cloud_host);
  if (c->counters_host) cudaFreeHost(c->counters_host);
  dfree(c->pt_route); dfree(c->vol_order); dfree(c->fld_c);
  dfree(c->poses); dfree(c->hits); dfree(c->sorted); dfree(c->sorted_n); dfree(c->dbg_tau); dfree(c->rank);
  dfree(c->n_hits);
  dfree(c->counts); dfree(c->offsets); dfree(c->S); dfree(c->S_raw); dfree(c->ptab); dfree(c->wtab); dfree(c->x_hi); dfree(c->x_lo); dfree(c->gain);
  dfree(c->sep_fz); dfree(c->ysep_hi); dfree(c->ysep_lo); dfree(c->taper_x_dev);
  dfree(c->env_stage); dfree(c->keys); dfree(c->pmax); dfree(c->cloud_stage); dfree(c->n_cloud_dev); dfree(c->err_dev); dfree(c->synth_bounds);
  auto& S = c->sur;
  dfree(S.params); dfree(S.wbf); dfree(S.wsmall); dfree(S.loss); dfree(S.feat); dfree(S.poses); dfree(S.buf); dfree(S.g);
  dfree(S.cmp_tot); dfree(S.cmp_pmax); dfree(S.cmp_pk); dfree(S.cmp_bmax);
  delete c;
  return SONAR_OK;
}

int sonar_scene_upload(sonar_ctx* ctx, const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                       const float* mu, const uint8_t* flags, const float* points, const float* sigma,
                       int64_t n_points, const double* planes, int64_t n_planes) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  if (n_verts < 0 || n_tris < 0 || n_points < 0 || n_planes < 0) return fail(ctx, SONAR_E_ARG, "negative count");
  if (n_tris > 0 && (!verts || !tris || !mu || !flags)) return fail(ctx, SONAR_E_ARG, "mesh arrays missing");
  if (n_points > 0 && (!points || !sigma)) return fail(ctx, SONAR_E_ARG, "point arrays missing");
  if (n_planes > 0 && !planes) return fail(ctx, SONAR_E_ARG, "plane array missing");
  if (n_tris >= (1LL << 30) || n_points >= (1LL << 23) || n_planes > 62)
    return fail(ctx, SONAR_E_UNSUPPORTED, "scene too large");
  for (int64_t i = 0; i < 3 * n_tris; ++i)
    if (tris[i] < 0 || tris[i] >= n_verts) return fail(ctx, SONAR_E_ARG, "triangle %lld has a bad vertex index", (long long)(i / 3));
  for (int64_t i = 0; i < 3 * n_verts; ++i)
    if (!isfinite(verts[i])) return fail(ctx, SONAR_E_ARG, "vertex %lld is not finite", (long long)(i / 3));
  CU(cudaSetDevice(ctx->device));
  int rc0 = drain(ctx);
  if (rc0) return rc0;
  CU(cudaStreamSynchronize(ctx->user_stream));
  CU(cudaStreamSynchronize(ctx->stream));
  free_scene(ctx);
  drop_graphs(ctx);
  if (n_tris > 0) {
    float* dv = nullptr;
    int32_t* dt = nullptr;
    float* dm = nullptr;
    uint8_t* df = nullptr;
    CU(cudaMalloc(&dv, sizeof(float) * 3 * n_verts));
    CU(cudaMalloc(&dt, sizeof(int32_t) * 3 * n_tris));
    CU(cudaMalloc(&dm, sizeof(float) * n_tris));
    CU(cudaMalloc(&df, n_tris));
    CU(cudaMemcpyAsync(dv, verts, sizeof(float) * 3 * n_verts, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(dt, tris, sizeof(int32_t) * 3 * n_tris, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(dm, mu, sizeof(float) * n_tris, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(df, flags, n_tris, cudaMemcpyHostToDevice, ctx->stream));
    cudaError_t e = build_bvh(dv, dt, verts, tris, ctx->bvh_opt == 0, dm, df, (int32_t)n_tris, &ctx->tri32, &ctx->triv,
                              &ctx->tri_prim, &ctx->tri_mu,
                              &ctx->tri_flags, &ctx->tri_plane, &ctx->tri_inv_n, &ctx->nodes, &ctx->sc.root,
                              ctx->stream);
    cudaFree(dv);
    cudaFree(dt);
    cudaFree(dm);
    cudaFree(df);
    CU(e);
  }
  if (n_points > 0) {
    std::vector<float4> pts(n_points);
    for (int64_t i = 0; i < n_points; ++i) pts[i] = make_float4(points[3 * i], points[3 * i + 1], points[3 * i + 2], sigma[i]);
    CU(cudaMalloc(&ctx->points, sizeof(float4) * n_points));
    CU(cudaMemcpy(ctx->points, pts.data(), sizeof(float4) * n_points, cudaMemcpyHostToDevice));
  }
  if (n_planes > 0) {
    CU(cudaMalloc(&ctx->planes, sizeof(double4_32a) * n_planes));
    CU(cudaMemcpy(ctx->planes, planes, sizeof(double4_32a) * n_planes, cudaMemcpyHostToDevice));
  }
  ctx->sc.tri32 = ctx->tri32;
  ctx->sc.triv = ctx->triv;
  ctx->sc.tri_prim = ctx->tri_prim;
  ctx->sc.tri_mu = ctx->tri_mu;
  ctx->sc.tri_flags = ctx->tri_flags;
  ctx->sc.tri_plane = ctx->tri_plane;
  ctx->sc.tri_plane_df = reinterpret_cast<const float4*>(ctx->tri_plane + n_tris);
  ctx->sc.tri_inv_n = ctx->tri_inv_n;
  ctx->sc.nodes = ctx->nodes;
  ctx->sc.n_tris = (int32_t)n_tris;
  ctx->sc.points = ctx->points;
  ctx->sc.n_points = (int32_t)n_points;
  ctx->sc.planes = ctx->planes;
  ctx->sc.n_planes = (int32_t)n_planes;
  ctx->has_scene = true;
  ctx->scene_version++;
  return SONAR_OK;
}

int sonar_ping(sonar_ctx* ctx, const sonar_pose* pose, const sonar_params* params, const sonar_ssp* ssp, float* env,
               sonar_point* cloud, int64_t cloud_cap, int64_t* n_cloud) {
  return run(ctx, pose, 1, params, ssp, env, cloud, cloud_cap, n_cloud);
}

int sonar_ping_batch(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings, const sonar_params* params,
                     const sonar_ssp* ssp, float* env, sonar_point* cloud, int64_t cloud_cap_per_ping,
                     int64_t* n_cloud) {
  return run(ctx, poses, n_pings, params, ssp, env, cloud, cloud_cap_per_ping, n_cloud);
}

int sonar_ping_async(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings, const sonar_params* params,
                     const sonar_ssp* ssp, float* env, sonar_point* cloud, int64_t cloud_cap_per_ping,
                     int64_t* n_cloud) {
  return run_async(ctx, poses, n_pings, params, ssp, env, cloud, cloud_cap_per_ping, n_cloud);
}

int sonar_wait(sonar_ctx* ctx) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  CU(cudaSetDevice(ctx->device));
  return drain(ctx);
}

int sonar_probe_wait_limit(sonar_ctx* ctx, int64_t limit_cycles) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  if (limit_cycles < 1 || limit_cycles > (1ll << 31)) return fail(ctx, SONAR_E_ARG, "limit_cycles lies outside 1 .. 2^31");
  CU(cudaSetDevice(ctx->device));
  const int rc = drain(ctx);
  if (rc) return rc;
  if (!ctx->err_dev) CU(cudaMalloc(&ctx->err_dev, sizeof(int)));
  CU(cudaMemsetAsync(ctx->err_dev, 0, sizeof(int), ctx->stream));
  k_wait_probe<<<1, 32, 0, ctx->stream>>>(ctx->err_dev, (long long)limit_cycles);
  CU(cudaGetLastError());
  int errw = 0;
  CU(cudaMemcpyAsync(&errw, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (errw & kErrTimeout) return fail(ctx, SONAR_E_TIMEOUT, "a device-side wait exceeded its limit");
  return SONAR_OK;
}

int sonar_get_hits(sonar_ctx* ctx, sonar_hit* out, int64_t cap, int64_t* n) {
  if (!ctx) return SONAR_E_ARG;
  {
    const int rc = drain(ctx);
    if (rc) return rc;
  }
  if (!ctx->debug) return fail(ctx, SONAR_E_ARG, "enable SONAR_OPT_DEBUG before the ping");
  if (ctx->last_p == 0) return fail(ctx, SONAR_E_ARG, "no ping yet");
  CU(cudaSetDevice(ctx->device));
  int64_t total = ctx->stats.n_hits;
  if (n) *n = total;
  int64_t k = total < cap ? total : cap;
  if (k > 0 && out) {
    std::vector<HitRec> h(k);
    std::vector<double> tau(k);
    CU(cudaMemcpyAsync(h.data(), ctx->hits, sizeof(HitRec) * k, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(tau.data(), ctx->dbg_tau, sizeof(double) * k, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int64_t i = 0; i < k; ++i) {
      out[i].key = h[i].key;
      out[i].prim = h[i].prim;
      out[i].tau = tau[i];
      out[i].amp = hypotf(h[i].cr, h[i].ci);
      out[i].phi = atan2f(h[i].ci, h[i].cr);
      out[i].uy = h[i].uy;
      out[i].uz = h[i].uz;
    }
  }
  if (total > cap) return fail(ctx, SONAR_E_CAPACITY, "%lld hits", (long long)total);
  return SONAR_OK;
}

int sonar_get_echoes(sonar_ctx* ctx, float* out, int64_t cap_floats) {
  if (!ctx || !out) return SONAR_E_ARG;
  {
    const int rc = drain(ctx);
    if (rc) return rc;
  }
  if (ctx->last_p == 0) return fail(ctx, SONAR_E_ARG, "no ping yet");
  const Derived& d = ctx->last_d;
  const int64_t per_ping = (int64_t)d.nr * d.M * 2;
  if (cap_floats < per_ping * ctx->last_p) return fail(ctx, SONAR_E_CAPACITY, "need %lld floats", (long long)(per_ping * ctx->last_p));
  CU(cudaSetDevice(ctx->device));
  // true-time delay: the wideband echoes at the range samples (phase 0)
  const float2* S = ctx->last_ttd_u > 0 ? ctx->S_raw : ctx->S;
  for (int p = 0; p < ctx->last_p; ++p) {
    const float2* src = S + ((int64_t)p * d.nr_pad + kPad) * d.M;
    CU(cudaMemcpyAsync(out + p * per_ping, src, sizeof(float) * per_ping, cudaMemcpyDeviceToHost, ctx->stream));
  }
  CU(cudaStreamSynchronize(ctx->stream));
  return SONAR_OK;
}

int sonar_get_raw(sonar_ctx* ctx, int32_t phase, float* out, int64_t cap_floats) {
  if (!ctx || !out) return SONAR_E_ARG;
  {
    const int rc = drain(ctx);
    if (rc) return rc;
  }
  if (ctx->last_p == 0 || ctx->last_raw_u == 0) return fail(ctx, SONAR_E_ARG, "no raw-series ping yet");
  if (!ctx->debug) return fail(ctx, SONAR_E_ARG, "enable SONAR_OPT_DEBUG before the ping");
  if (phase < 0 || phase >= ctx->last_raw_u) return fail(ctx, SONAR_E_ARG, "phase %d outside [0, %d)", phase, ctx->last_raw_u);
  const Derived& d = ctx->last_d;
  const int64_t per_ping = (int64_t)d.nr * d.M * 2;
  if (cap_floats < per_ping * ctx->last_p) return fail(ctx, SONAR_E_CAPACITY, "need %lld floats", (long long)(per_ping * ctx->last_p));
  CU(cudaSetDevice(ctx->device));
  for (int p = 0; p < ctx->last_p; ++p) {
    const float2* src = ctx->S_raw + (int64_t)phase * ctx->s_elems + ((int64_t)p * d.nr_pad + kPad) * d.M;
    CU(cudaMemcpyAsync(out + p * per_ping, src, sizeof(float) * per_ping, cudaMemcpyDeviceToHost, ctx->stream));
  }
  CU(cudaStreamSynchronize(ctx->stream));
  return SONAR_OK;
}

int sonar_get_stats(const sonar_ctx* ctx, sonar_stats* out) {
  if (!ctx || !out) return SONAR_E_ARG;
  *out = ctx->stats;
  return SONAR_OK;
}


int sonar_sur_set_weights(sonar_ctx* ctx, const float* params, int64_t n, double e_scale) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  if (!params || n != kSurParams) return fail(ctx, SONAR_E_ARG, "need %lld parameters", (long long)kSurParams);
  if (!(e_scale > 0) || !isfinite(e_scale)) return fail(ctx, SONAR_E_ARG, "e_scale must be positive");
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(params[i])) return fail(ctx, SONAR_E_ARG, "parameter %lld is not finite", (long long)i);
  CU(cudaSetDevice(ctx->device));
  int rc;
  if ((rc = drain(ctx))) return rc;
  if ((rc = sur_alloc_params(ctx))) return rc;
  auto& S = ctx->sur;
  CU(cudaMemcpyAsync(S.net.theta, params, sizeof(float) * kSurParams, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaMemsetAsync(S.net.m, 0, sizeof(float) * 2 * kSurParams, ctx->stream));
  CU(sur_pack(S.net, 0, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  S.e_scale = e_scale;
  S.step = 0;
  S.has_weights = true;
  return SONAR_OK;
}

int sonar_sur_get_weights(sonar_ctx* ctx, float* params, int64_t n) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  if (!params || n != kSurParams) return fail(ctx, SONAR_E_ARG, "need room for %lld parameters", (long long)kSurParams);
  if (!ctx->sur.has_weights) return fail(ctx, SONAR_E_ARG, "the surrogate has no weights");
  CU(cudaSetDevice(ctx->device));
  CU(cudaStreamSynchronize(ctx->stream));
  CU(cudaMemcpy(params, ctx->sur.net.theta, sizeof(float) * kSurParams, cudaMemcpyDeviceToHost));
  return SONAR_OK;
}

int sonar_sur_render(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings, const sonar_params* params,
                     const sonar_ssp* ssp, float* feat) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  if (!feat) return fail(ctx, SONAR_E_ARG, "feat is NULL");
  Derived d;
  const bool had = ctx->sur.has_weights;
  ctx->sur.has_weights = true;  // the rendering needs no network
  int rc = sur_begin(ctx, poses, n_pings, params, ssp, d);
  ctx->sur.has_weights = had;
  if (rc) return rc;
  const int64_t n = (int64_t)n_pings * d.nb * 8;
  void* fd = nullptr;
  if (classify(feat, &fd) != Mem::Host) {
    CU(cudaMemcpyAsync(fd, ctx->sur.feat, sizeof(float) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    return sur_finish(ctx);
  }
  if ((rc = sur_finish(ctx))) return rc;
  CU(cudaMemcpy(feat, ctx->sur.feat, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return SONAR_OK;
}

int sonar_sur_ping(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings, const sonar_params* params,
                   const sonar_ssp* ssp, float* env) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  if (!env) return fail(ctx, SONAR_E_ARG, "env is NULL");
  Derived d;
  int rc = sur_begin(ctx, poses, n_pings, params, ssp, d);
  if (rc) return rc;
  const int64_t beams = (int64_t)n_pings * d.nb;
  const int64_t chunk = beams < kSurChunk ? beams : kSurChunk;
  if ((rc = sur_buffers(ctx, chunk, d.nr + 2 * kSurHalo))) return rc;
  void* ed = nullptr;
  const bool dev = classify(env, &ed) != Mem::Host;
  float* out = static_cast<float*>(ed);
  if (!dev) {
    if ((rc = grow(ctx, ctx->env_stage, ctx->env_cap, beams * d.nr, sizeof(float), false))) return rc;
    out = ctx->env_stage;
  }
  for (int64_t b0 = 0; b0 < beams; b0 += chunk) {
    const int64_t nb = beams - b0 < chunk ? beams - b0 : chunk;
    if ((rc = sur_forward(ctx, ctx->sur.feat + b0 * 8, nullptr, nb, nb, params, d, nullptr, out + b0 * d.nr)))
      return rc;
  }
  if ((rc = sur_finish(ctx))) return rc;
  if (!dev) CU(cudaMemcpy(env, ctx->env_stage, sizeof(float) * beams * d.nr, cudaMemcpyDeviceToHost));
  return SONAR_OK;
}

int sonar_sur_geometric(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings, const sonar_params* params,
                        const sonar_ssp* ssp, float* env) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  if (!env) return fail(ctx, SONAR_E_ARG, "env is NULL");
  Derived d;
  const bool had = ctx->sur.has_weights;
  ctx->sur.has_weights = true;  // no network involved
  int rc = sur_begin(ctx, poses, n_pings, params, ssp, d);
  ctx->sur.has_weights = had;
  if (rc) return rc;
  if ((rc = ensure_tables(ctx, params, d))) return rc;
  const int64_t beams = (int64_t)n_pings * d.nb;
  void* ed = nullptr;
  const bool dev = classify(env, &ed) != Mem::Host;
  float* out = static_cast<float*>(ed);
  if (!dev) {
    if ((rc = grow(ctx, ctx->env_stage, ctx->env_cap, beams * d.nr, sizeof(float), false))) return rc;
    out = ctx->env_stage;
  }
  CU(sur_geometric(ctx->sur.feat, beams, params->n_beam_az, params->n_beam_el, params->hfov_rad, params->vfov_rad, d.nr,
                   params->r_min_m, d.dr, d.c_ref, params->alpha_np_per_m, params->pulse_s, ctx->rtab, kRTab, out,
                   ctx->stream));
  if ((rc = sur_finish(ctx))) return rc;
  if (!dev) CU(cudaMemcpy(env, ctx->env_stage, sizeof(float) * beams * d.nr, cudaMemcpyDeviceToHost));
  return SONAR_OK;
}

int sonar_sur_train_step(sonar_ctx* ctx, const sonar_pose* poses, int32_t n_pings, const sonar_params* params,
                         const sonar_ssp* ssp, const float* env_target, const int32_t* beams, int64_t n_sel,
                         double lr, int32_t update, double* loss, float* grad) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  if (!env_target) return fail(ctx, SONAR_E_ARG, "env_target is NULL");
  if (update && !(lr > 0 && isfinite(lr))) return fail(ctx, SONAR_E_ARG, "lr must be positive");
  Derived d;
  int rc = sur_begin(ctx, poses, n_pings, params, ssp, d);
  if (rc) return rc;
  const int64_t n_feat = (int64_t)n_pings * d.nb;
  if (!beams) n_sel = n_feat;
  if (n_sel < 1 || n_sel > (1LL << 24)) return fail(ctx, SONAR_E_ARG, "n_sel must lie in [1, 2^24]");
  void* td = nullptr;
  void* bd = nullptr;
  if (classify(const_cast<float*>(env_target), &td) == Mem::Host)
    return fail(ctx, SONAR_E_ARG, "env_target must be device memory");
  if (beams && classify(const_cast<int32_t*>(beams), &bd) == Mem::Host)
    return fail(ctx, SONAR_E_ARG, "beams must be device memory");
  auto& S = ctx->sur;
  if ((rc = sur_buffers(ctx, n_sel, d.nr + 2 * kSurHalo))) return rc;
  if ((rc = grow(ctx, S.g, S.g_cap, n_sel * d.nr, sizeof(float), false))) return rc;
  CU(cudaMemsetAsync(S.net.grad, 0, sizeof(float) * kSurParams, ctx->stream));
  CU(cudaMemsetAsync(S.loss, 0, sizeof(double), ctx->stream));
  const int32_t* bsel = static_cast<const int32_t*>(bd);
  if ((rc = sur_forward(ctx, S.feat, bsel, n_sel, n_feat, params, d, static_cast<const float*>(td), nullptr))) return rc;
  if ((rc = sur_backward(ctx, S.feat, bsel, n_sel, n_feat, params, d))) return rc;
  if (update) {
    const double b1 = 0.9, b2 = 0.999;
    const int64_t t = S.step + 1;
    CU(sur_pack(S.net, 1, (float)lr, (float)b1, (float)b2, 1e-8f, (float)(1.0 - pow(b1, (double)t)),
                (float)(1.0 - pow(b2, (double)t)), ctx->stream));
  }
  if ((rc = sur_finish(ctx))) return rc;
  if (update) S.step++;
  if (loss) {
    double sq = 0.0;
    CU(cudaMemcpy(&sq, S.loss, sizeof(double), cudaMemcpyDeviceToHost));
    *loss = sq / ((double)n_sel * d.nr);
  }
  if (grad) CU(cudaMemcpy(grad, S.net.grad, sizeof(float) * kSurParams, cudaMemcpyDeviceToHost));
  return SONAR_OK;
}

int sonar_sur_compare(sonar_ctx* ctx, const float* env, const float* env_ref, int32_t n_pings,
                      const sonar_params* params, double rel_thr, sonar_sur_metrics* out) {
  if (!ctx) return SONAR_E_ARG;
  ctx->err.clear();
  if (!env || !env_ref || !out || n_pings < 1 || !params) return fail(ctx, SONAR_E_ARG, "bad arguments");
  if (!(rel_thr >= 0 && rel_thr <= 1)) return fail(ctx, SONAR_E_ARG, "rel_thr must lie in [0, 1]");
  if (params->n_beam_az < 1 || params->n_beam_el < 1 || params->n_range < 1 || !(params->r_max_m > params->r_min_m))
    return fail(ctx, SONAR_E_ARG, "bad beam or range grid");
  void* ed = nullptr;
  void* rd = nullptr;
  if (classify(const_cast<float*>(env), &ed) == Mem::Host || classify(const_cast<float*>(env_ref), &rd) == Mem::Host)
    return fail(ctx, SONAR_E_ARG, "both volumes must be device memory");
  CU(cudaSetDevice(ctx->device));
  int rc;
  if ((rc = drain(ctx))) return rc;
  auto& S = ctx->sur;
  const int nb = params->n_beam_az * params->n_beam_el, nr = params->n_range;
  const int64_t beams = (int64_t)n_pings * nb;
  if (!S.cmp_tot) CU(cudaMalloc(&S.cmp_tot, sizeof(double) * 12));
  if ((rc = grow(ctx, S.cmp_pmax, S.cmp_cap, n_pings, sizeof(unsigned), false))) return rc;
  if ((rc = grow(ctx, S.cmp_pk, S.cmp_pk_cap, 2 * beams, sizeof(int32_t), false))) return rc;
  if ((rc = grow(ctx, S.cmp_bmax, S.cmp_bmax_cap, beams, sizeof(float), false))) return rc;
  const double dr = (params->r_max_m - params->r_min_m) / nr;
  int n_blank = 0;
  while (n_blank < nr && params->r_min_m + (n_blank + 0.5) * dr < params->r_blank_m) ++n_blank;
  CU(cudaEventRecord(ctx->ev_in, ctx->user_stream));
  CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
  CU(cudaMemsetAsync(S.cmp_tot, 0, sizeof(double) * 12, ctx->stream));
  CU(cudaMemsetAsync(S.cmp_pmax, 0, sizeof(unsigned) * n_pings, ctx->stream));
  CU(sur_compare(static_cast<const float*>(ed), static_cast<const float*>(rd), n_pings, nb, nr, n_blank, (float)rel_thr,
                 S.cmp_pmax, S.cmp_pk, S.cmp_bmax, S.cmp_tot, ctx->stream));
  CU(cudaEventRecord(ctx->ev_out, ctx->stream));
  CU(cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0));
  CU(cudaStreamSynchronize(ctx->stream));
  double t[12];
  CU(cudaMemcpy(t, S.cmp_tot, sizeof(t), cudaMemcpyDeviceToHost));
  out->nl2 = t[1] > 0 ? sqrt(t[0] / t[1]) : 0.0;
  out->lit_beams = (int64_t)t[3];
  out->peak_bin_mean = t[3] > 0 ? t[2] / t[3] : 0.0;
  out->peak_within_1 = t[3] > 0 ? t[4] / t[3] : 0.0;
  out->peak_within_4 = t[3] > 0 ? t[5] / t[3] : 0.0;
  out->cells = (int64_t)t[6];
  const double m1 = t[6] > 0 ? t[7] / t[6] : 0.0, m2 = t[6] > 0 ? t[8] / t[6] : 0.0;
  const double r1 = t[6] > 0 ? t[9] / t[6] : 0.0, r2 = t[6] > 0 ? t[10] / t[6] : 0.0;
  out->si = m1 > 0 ? m2 / (m1 * m1) - 1.0 : 0.0;
  out->si_ref = r1 > 0 ? r2 / (r1 * r1) - 1.0 : 0.0;
  return SONAR_OK;
}
}  // extern "C"
