// Phase-shift beamforming (Sec. II.B coherent summation into beams) as one dense
// contraction on the 5th-generation tensor cores, with the envelope, time-varied gain
// and per-beam peak search fused into the epilogue.
//
// Complex B[b][n] = sum_m W[b][m] s_m[n] is run as a real GEMM
//   C[n][2b + r] = sum_k X[n][k] Y[2b + r][k],  k = 2m + c,
// X = element echoes with (re, im) interleaved per element (K-major), and Y the static
// real 4-form of the steering matrix: row 2b = (Wr, -Wi) pairs, row 2b+1 = (Wi, Wr).
// A thread of the epilogue then holds (Re, Im) of a beam in adjacent accumulator
// columns. Tiles: 128 range samples x (tile_n / 2) beams, K step 64 (one 128-byte
// swizzle atom), operands staged by TMA into a 4-stage ring, MMAs issued by one thread
// into a double-buffered TMEM accumulator (2 x tile_n columns) so the epilogue of one
// tile overlaps the MMAs of the next. Persistent CTAs, one per SM.
//
// Operand delivery bounds the contraction: every tile streams its A rows (128) and B
// rows (tile_n) from L2, about 14 TB/s over all SMs. With a number of row tiles that CS
// (2 or 4) divides, the CTAs run in clusters of CS that take CS row tiles of the same N
// tile together: each loads its own A tile and 1 / CS of the shared B tile, multicast
// into every CTA's stages, so a tile moves 128 + tile_n / CS rows instead of 128 +
// tile_n. A stage is refilled only after all CS CTAs' MMAs have released it (their
// commits arrive on every CTA's empty barriers), and a cluster barrier brackets the
// kernel so that no CTA leaves while a peer may still write into its shared memory.
//
// FP32 form: X = Xh + Xl, Y = Yh + Yl in BF16; the three products hi*hi, hi*lo, lo*hi
// accumulate into the same FP32 accumulator. Its stages hold all four operand tiles of a
// 32-deep K slice (64-byte swizzle) and issue the three products from them: each tile
// crosses shared memory once instead of twice, which matters because an M = 128 MMA on
// one SM is bound by shared-memory bandwidth (operand reads plus TMA writes), while four
// stages keep the pipeline as deep as the one-product forms' 64-deep, two-tile stages.
#include <math.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace sonar {
namespace {
using namespace tc;

constexpr int BM = 128;
#ifndef SONAR_GEMM_EPI_WARPS
#define SONAR_GEMM_EPI_WARPS 16
#endif
// warp 0 TMA, warp 1 MMA, then the epilogue warps: kEpiWarps / 4 per TMEM lane quarter,
// each taking every (kEpiWarps / 4)-th 32-column chunk of the tile, so that a tile's
// drain keeps pace with the MMAs of the next (it bounds the one-product forms, whose
// MMAs per tile are short)
constexpr int kEpiWarps = SONAR_GEMM_EPI_WARPS;
static_assert(kEpiWarps % 4 == 0, "epilogue warps come in lane-quarter sets of four");
constexpr int kGemmThreads = 32 * (2 + kEpiWarps);

// NPASS products per K slice (1: BF16/FP16, 3: FP32 form); PARTS tiles per operand (hi,
// lo) in a stage; BK the K slice (64: 128-byte swizzle, 32: 64-byte swizzle).
template <int NPASS, int BN = 224>
struct GemmShape {
  static constexpr int PARTS = NPASS == 3 ? 2 : 1;
  static constexpr int BK = NPASS == 3 ? 32 : 64;
  // as many stages as 224 KB of shared memory hold, up to five
  static constexpr int STAGE_BYTES = PARTS * (BM + BN) * BK * 2;
  static constexpr int STAGES = (224 * 1024) / STAGE_BYTES < 5 ? (224 * 1024) / STAGE_BYTES : 5;
};

// UMMA shared-memory descriptor, K-major, 64-byte swizzle: 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// TMEM columns of the double-buffered accumulator: 2 BN rounded up to a power of two
// (allocation granularity).
constexpr uint32_t tmem_cols(int bn) { return 2 * bn <= 256 ? 256u : 512u; }


// Tile order: groups of up to 16 row tiles; inside a group the column tiles run in
// the outer loop, so concurrently running CTAs share one steering block through L2.
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int& mb, int& nb) {
  const int G = 16;
  int group = t / (G * tiles_n);
  int gm0 = group * G;
  int gsz = min(G, tiles_m - gm0);
  int r = t - group * G * tiles_n;
  nb = r / gsz;
  mb = gm0 + r % gsz;
}

// One beam of a drained chunk: the envelope sqrt(re^2 + im^2) x scale, stored when
// `store`; over the warp's eligible samples the maximum m (a warp reduction of the
// value bits, which order like the values since e >= 0) and the ballot of the lanes
// holding it; lane j keeps both, and pmax follows m.
__device__ __forceinline__ void epi_beam(uint32_t vre, uint32_t vim, float scale, float* dst, bool store, bool elig,
                                         int j, int lane, uint32_t& km, uint32_t& kbal, uint32_t& pmax) {
  const float re = __uint_as_float(vre), im = __uint_as_float(vim);
  // sqrt.approx: relative error below 2^-22, a fraction of the BF16 hi/lo operands' 2^-17
  // (the rounded square root's slow path was a third of a short contraction's time)
  float e;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(e) : "f"(fmaf(re, re, im * im)));
  e *= scale;
  if (store) *dst = e;
  const uint32_t eb = __float_as_uint(e);
  const uint32_t m = __reduce_max_sync(0xffffffffu, elig ? eb : 0u);
  const uint32_t at = __ballot_sync(0xffffffffu, elig && eb == m);
  if (lane == j) {
    km = m;
    kbal = at;
  }
  pmax = max(pmax, m);
}

template <int BN, int NPASS, int CS>
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm(const __grid_constant__ GemmArgs a, uint32_t idesc) {
  constexpr bool MC = CS > 1;
  constexpr uint16_t kMask = (uint16_t)((1u << CS) - 1u);
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // align by pointer arithmetic on the shared array, so that the compiler keeps the
  // shared address space (an integer round trip would turn every access generic)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  constexpr int PARTS = GemmShape<NPASS, BN>::PARTS, BK = GemmShape<NPASS, BN>::BK;
  constexpr int STAGES = GemmShape<NPASS, BN>::STAGES;
  constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
  uint8_t* sA = smem;                                 // [stage][part] A tiles (X: echoes)
  uint8_t* sB = smem + STAGES * PARTS * A_BYTES;      // [stage][part] B tiles (Y: steering)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + STAGES * PARTS * B_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* tfull = bars + 2 * STAGES;
  uint64_t* tempty = bars + 2 * STAGES + 2;
  uint64_t* done = bars + 2 * STAGES + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = a.tiles_m * a.tiles_n;
  const int k_iters = a.k_blocks * (64 / BK);  // K slices per tile
  // work units: tiles, or (clusters of CS) groups of CS row tiles of one N tile
  const int rank = MC ? (int)cluster_rank() : 0;
  const int n_units = n_tiles / CS;
  const int unit0 = (int)blockIdx.x / CS;
  const int ustep = (int)gridDim.x / CS;
  auto coords = [&](int u, int& mb, int& nb) {
    int mbg;
    tile_coords(u, a.tiles_m / CS, a.tiles_n, mbg, nb);
    mb = CS * mbg + rank;
  };
  constexpr uint32_t B_PART = B_BYTES / CS;  // one CTA's share of a B tile (tile_n / CS rows)

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), CS);  // released by every CTA's MMAs
    }
    for (int s = 0; s < 2; ++s) { mbar_init(smem_u32(&tfull[s]), 1); mbar_init(smem_u32(&tempty[s]), kEpiWarps); }
    mbar_init(smem_u32(done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols(BN)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  if (MC) cluster_sync();  // the peers' barriers are initialised before anything reaches them
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // the operands come from the conversion kernel
  pdl_wait();

  if (warp == 0) {
    // ------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued = 0;
      bool ok = true;
      for (int u = unit0; u < n_units && ok; u += ustep) {
        int mb, nb;
        coords(u, mb, nb);
        // the tile's first X row: ping p's block of x_ping_rows rows, past its guard rows
        const int row0 = mb * BM, p = row0 / a.nr_x;
        const int y_tile = p * a.x_ping_rows + a.x_guard + (row0 - p * a.nr_x);
        int xk = 0, lvl = 0, y = y_tile;  // K position inside the level, the level, its X row
        // separable beams: the block of the tile's elevation row
        if (a.sep_az > 0) y += (int)((int64_t)nb * (BN / 2) / a.sep_az * a.x_el_rows);
        if (a.ttd_u > 0) {
          const int q = a.ttd_q0, s = ((q % a.ttd_u) + a.ttd_u) % a.ttd_u;
          y = y_tile + s * a.x_phase_rows + (q - s) / a.ttd_u;
        }
        for (int kb = 0; kb < k_iters && ok; ++kb) {
          if (!mbar_wait(smem_u32(&empty[stage]), phase ^ 1, a.err)) { ok = false; break; }
          const uint32_t fb = smem_u32(&full[stage]);
          mbar_expect_tx(fb, PARTS * (A_BYTES + B_BYTES));
          uint8_t* const a_st = sA + stage * PARTS * A_BYTES;
          uint8_t* const b_st = sB + stage * PARTS * B_BYTES;
          tma_load_2d(smem_u32(a_st), &a.map_xh, xk, y, fb);
          if (MC) tma_load_2d_mc(smem_u32(b_st) + rank * B_PART, &a.map_yh, kb * BK, nb * BN + rank * (BN / CS), fb, kMask);
          else tma_load_2d(smem_u32(b_st), &a.map_yh, kb * BK, nb * BN, fb);
          if (PARTS == 2) {
            tma_load_2d(smem_u32(a_st + A_BYTES), &a.map_xl, xk, y, fb);
            if (MC)
              tma_load_2d_mc(smem_u32(b_st + B_BYTES) + rank * B_PART, &a.map_yl, kb * BK, nb * BN + rank * (BN / CS),
                             fb, kMask);
            else tma_load_2d(smem_u32(b_st + B_BYTES), &a.map_yl, kb * BK, nb * BN, fb);
          }
          xk += BK;
          if (xk == a.x_kpad && a.ttd_u > 0) {
            // next fractional-delay level: phase q mod U, row offset floor(q / U)
            xk = 0;
            const int q = a.ttd_q0 + (++lvl), s = ((q % a.ttd_u) + a.ttd_u) % a.ttd_u;
            y = y_tile + s * a.x_phase_rows + (q - s) / a.ttd_u;
          }
          ++issued;
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
      }
      if (!ok) {
        // wait (bounded) for copies still in flight before the CTA exits
        for (int j = 0; j < STAGES && j < issued; ++j) {
          if (--stage < 0) { stage = STAGES - 1; phase ^= 1; }
          mbar_wait(smem_u32(&full[stage]), phase, a.err);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      for (int u = unit0; u < n_units && ok; u += ustep) {
        if (!mbar_wait(smem_u32(&tempty[acc]), acc_phase ^ 1, a.err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
        for (int it = 0; it < k_iters; ++it) {
          if (!mbar_wait(smem_u32(&full[stage]), phase, a.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ah = smem_u32(sA + stage * PARTS * A_BYTES), bh = smem_u32(sB + stage * PARTS * B_BYTES);
#pragma unroll
          for (int pass = 0; pass < NPASS; ++pass) {
            // hi*hi, then hi*lo, then lo*hi; a K step of 16 advances 32 bytes in the row
            const uint32_t a0 = pass == 2 ? ah + A_BYTES : ah, b0 = pass == 1 ? bh + B_BYTES : bh;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint64_t da = BK == 64 ? sw128_desc(a0 + kk * 32) : sw64_desc(a0 + kk * 32);
              const uint64_t db = BK == 64 ? sw128_desc(b0 + kk * 32) : sw64_desc(b0 + kk * 32);
              tc_mma(d_tmem, da, db, idesc, (it | pass | kk) != 0);
            }
          }
          if (MC) tc_commit_mc(smem_u32(&empty[stage]), kMask);
          else tc_commit(smem_u32(&empty[stage]));
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        tc_commit(smem_u32(&tfull[acc]));
        if (++acc == 2) { acc = 0; acc_phase ^= 1; }
      }
      // all issued MMAs complete before TMEM is released
      tc_commit(smem_u32(done));
      mbar_wait(smem_u32(done), 0, a.err);
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int sub = (warp - 2) >> 2;  // chunks sub, sub + kEpiWarps / 4, ...
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int u = unit0; u < n_units; u += ustep) {
      int mb, nb;
      coords(u, mb, nb);
      if (!mbar_wait(smem_u32(&tfull[acc]), acc_phase, a.err)) break;
      tc_fence_after();
      const int row = mb * BM + q * 32 + lane;
      const int p = row / a.nr_x, n = row % a.nr_x;
      const bool vn = n < a.nr;
      const bool elig = vn && n >= a.n_blank;
      const float r = a.r_min + ((float)n + 0.5f) * a.dr;
      const float scale = r * __expf(a.alpha2 * r) * a.y_gain_inv / (a.gain ? a.gain[p] : 1.0f);
      float* env_p = a.env + (size_t)p * a.n_beams * a.nr;
      unsigned long long* keys_p = a.peak_keys + (size_t)p * a.n_beams;
      const int n0 = n - lane;  // the warp's rows: samples n0 .. n0 + 31 of ping p (nr_x is a multiple of 128)
      uint32_t pmax = 0u;       // the warp's maximum over its eligible entries (float bits, e >= 0)
#pragma unroll 1
      for (int c = sub; c < BN / 32; c += kEpiWarps / 4) {
        uint32_t v[32];
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c * 32);
        TMEM_LD_32(taddr, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // 16 beams: envelope, store, and per beam the warp's maximum over its 32 samples
        // (lane j < 16 keeps beam j's); one atomic per beam
        const int beam0 = nb * (BN / 2) + c * 16;
        float* dst = env_p + (size_t)beam0 * a.nr + n;
        uint32_t km = 0u, kbal = 0u;
        if (beam0 + 16 <= a.n_beams) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            epi_beam(v[2 * j], v[2 * j + 1], scale, dst + (size_t)j * a.nr, vn, elig, j, lane, km, kbal, pmax);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const bool vb = beam0 + j < a.n_beams;
            epi_beam(v[2 * j], v[2 * j + 1], scale, dst + (size_t)j * a.nr, vn && vb, elig && vb, j, lane, km, kbal,
                     pmax);
          }
        }
        // key: value bits over the complement of the first sample holding the maximum, so
        // that the larger key is the larger value and, among equal values, the earlier bin
        if (kbal != 0u)
          atomicMax(&keys_p[beam0 + lane], ((unsigned long long)km << 32) |
                                               (unsigned long long)(0xFFFFFFFFu - (uint32_t)(n0 + __ffs(kbal) - 1)));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&tempty[acc]));
        atomicMax(&a.ping_max[p], pmax);
      }
      if (++acc == 2) { acc = 0; acc_phase ^= 1; }
    }
  }
  tc_fence_before();
  if (MC) cluster_sync();  // no peer writes into this CTA's stages or barriers any more
  else __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols(BN)) : "memory");
  }
}

template <int BN, int NPASS>
constexpr size_t gemm_smem() {
  return 1024 + (size_t)GemmShape<NPASS, BN>::STAGES * GemmShape<NPASS, BN>::STAGE_BYTES + 256;
}
static_assert(gemm_smem<256, 3>() <= 227 * 1024 && gemm_smem<256, 1>() <= 227 * 1024, "GEMM stages fit");

// ----------------------------------------------------------------- steering matrix
// W[b][m] = w_m exp(-j k_a u_b . p_m) / sum w, beams cell-centred (Sec. III Eq. 2-3),
// scaled by `gain`; phase in FP64 cycles reduced modulo one before the FP32 sincos. The
// beam directions come from a per-beam table (FP64 trigonometry once per beam, not once
// per entry: FP64 transcendentals are slow on this part).
// With true-time delay (ttd != 0) the columns form n_levels blocks of k_pad, one per
// fractional-delay level q = q0 + block, each entry weighted by the 4-point Lagrange
// kernel h(x - q) at the pair's steering delay x (units of dt / U).
__device__ __forceinline__ double lagrange4(double y) {
  const double t = fabs(y);
  if (t < 1.0) return (t * t - 1.0) * (t - 2.0) * 0.5;
  if (t < 2.0) return -(t - 1.0) * (t - 2.0) * (t - 3.0) / 6.0;
  return 0.0;
}

__global__ void k_steer(SteerArgs a) {
  const int64_t rows = 2LL * a.nb_pad;
  const int64_t cols = (int64_t)a.n_levels * a.k_pad;
  const int64_t total = rows * cols;
  const int M = a.nx * a.ny, Nb = a.n_beam_az * a.n_beam_el;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i / cols;
    const int64_t kk = i - j * cols;
    const int lvl = (int)(kk / a.k_pad);
    const int k = (int)(kk - (int64_t)lvl * a.k_pad);
    const int b = (int)(j / 2), part = (int)(j % 2);
    const int m = k / 2, cpart = k % 2;
    float val = 0.f;
    if (b < Nb && m < M) {
      const double2 u = a.beam_uyz[b];  // the beam centre's direction cosines, once per beam
      const double uy = u.x, uz = u.y;
      const int mx = m % a.nx, my = m / a.nx;
      const double up = (mx - 0.5 * (a.nx - 1)) * uy + (my - 0.5 * (a.ny - 1)) * uz;
      const double cyc = a.pitch_over_lambda * up;
      const double fr = cyc - floor(cyc);
      float s, c;
      sincospif((float)(2.0 * fr), &s, &c);
      double w = (a.taper ? (double)a.taper[m] : 1.0) / a.wsum * a.gain;
      if (a.ttd) w *= lagrange4(-a.x_scale * up - (double)(a.q0 + lvl));
      const float wr = (float)(w * c), wi = (float)(-w * s);  // W = w e^{-j phi}
      if (part == 0) val = cpart == 0 ? wr : -wi;
      else val = cpart == 0 ? wi : wr;
    }
    if (a.mode == SONAR_FP16) {
      reinterpret_cast<__half*>(a.y_hi)[i] = __float2half_rn(val);
    } else {
      __nv_bfloat16 hi = __float2bfloat16_rn(val);
      reinterpret_cast<__nv_bfloat16*>(a.y_hi)[i] = hi;
      if (a.mode == SONAR_FP32)
        reinterpret_cast<__nv_bfloat16*>(a.y_lo)[i] = __float2bfloat16_rn(val - __bfloat162float(hi));
    }
  }
}

// ----------------------------------------------------------------- peaks -> cloud
// Per ping: decode each beam's packed (value, first index) maximum, apply the absolute
// or ping-relative threshold, and write points in beam order. One CTA per 1024 beams of a
// ping: it recounts the kept beams of the chunks before its own (a few thousand keys, so
// no CTA waits on another), then places its own by a block-wide exclusive scan of the
// keep flags. Positions in FP32 (a 15 m range keeps them within ~1e-6 m), from the
// beam grid and pose rounded to FP32 once (FP64 work per thread is slow on this part).
__device__ __forceinline__ bool peak_kept(unsigned long long key, float thr) {
  return key != 0ull && __uint_as_float((uint32_t)(key >> 32)) >= thr;
}

__global__ void __launch_bounds__(1024) k_peaks(PeakArgs a) {
  __shared__ int s_warp[32];
  pdl_wait();
  __shared__ int s_before;
  const int p = blockIdx.y, chunk = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int Nb = a.n_beam_az * a.n_beam_el;
  const float vmax = __uint_as_float(a.ping_max[p]);
  const float thr = a.thr_mode == 1 ? a.thr * vmax : a.thr;
  const unsigned long long* keys = a.peak_keys + (size_t)p * Nb;
  const int b0 = chunk * 1024;
  // this thread's beam, and the kept beams in the chunks before this one: independent
  // loads, issued together (eight at a time)
  const int b = b0 + t;
  const unsigned long long key = b < Nb ? __ldg(&keys[b]) : 0ull;
  int before = 0;
#pragma unroll 8
  for (int j = 0; j < chunk; ++j) before += peak_kept(__ldg(&keys[j * 1024 + t]), thr) ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
  if (lane == 0) s_warp[wid] = before;
  __syncthreads();
  if (wid == 0) {
    int v = s_warp[lane];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_before = v;
  }
  __syncthreads();
  const int base = s_before;
  // this chunk: exclusive scan of the keep flags
  const bool keep = peak_kept(key, thr);
  const unsigned ballot = __ballot_sync(0xffffffffu, keep);
  const int in_warp = __popc(ballot & ((1u << lane) - 1u));
  __syncthreads();  // s_warp is reused
  if (lane == 0) s_warp[wid] = __popc(ballot);
  __syncthreads();
  if (wid == 0) {
    const int v = s_warp[lane];
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_warp[lane] = x - v;  // exclusive prefix of warp counts
  }
  __syncthreads();
  const long long pos = (long long)base + s_warp[wid] + in_warp;
  if (keep && pos < a.cap) {
    const float* R = a.poses[p].R32;
    const float* T = a.poses[p].t32;
    const int n = (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
    const int bi = b % a.n_beam_az, bj = b / a.n_beam_az;
    float saz, caz, sel, cel;
    sincosf(a.az0 + ((float)bi + 0.5f) * a.daz, &saz, &caz);
    sincosf(a.el0 + ((float)bj + 0.5f) * a.del, &sel, &cel);
    const float r = a.r_min + ((float)n + 0.5f) * a.dr;
    const float v0 = r * cel * caz, v1 = r * cel * saz, v2 = r * sel;
    sonar_point pt;
    pt.x = R[0] * v0 + R[1] * v1 + R[2] * v2 + T[0];
    pt.y = R[3] * v0 + R[4] * v1 + R[5] * v2 + T[1];
    pt.z = R[6] * v0 + R[7] * v1 + R[8] * v2 + T[2];
    pt.intensity = __uint_as_float((uint32_t)(key >> 32));
    pt.beam = b;
    pt.bin = n;
    a.cloud[(size_t)p * a.cap + pos] = pt;
  }
  // the last chunk knows the ping's total
  if (chunk == gridDim.x - 1 && t == 1023) {
    a.n_cloud[p] = pos + (keep ? 1 : 0);
    a.n_cloud_host[p] = pos + (keep ? 1 : 0);
  }
  // every earlier kernel of the call has completed (the dependent-launch chain)
  if (p == 0 && chunk == 0 && t == 0) {
    a.counters_host[0] = a.n_hits[0];
    a.counters_host[1] = (unsigned long long)(unsigned)*a.err;
    a.counters_host[2] = a.n_hits[1];
  }
}

// ----------------------------------------------------------------- separable beams, stage 1
// U[el][n][mx] = sum_my Fz[el][my] s_(my, mx)[n], in units of kSepRows (two) range
// samples of one ping. Persistent CTAs (two per SM) hold Fz (as quads) in shared memory
// and take the units in turn; the two S rows of the next unit arrive by one bulk copy into
// the other half of a double buffer while the current unit is summed, so that the copy's
// latency and the CTA's prologue are paid once, not per unit. Lane mx of warp w
// accumulates eight elevations for both samples, each complex multiply-add two packed
// FP32 operations. Lanes past nx write zero columns, so the whole 64-column operand row is
// defined.
constexpr int kSepRows = 2;
constexpr int kSepMaxFz = 4096;  // n_el x ny entries of Fz held in shared memory
constexpr int kSepLd = 8;        // 16-byte loads per thread in flight at once (Fz staging)

__device__ __forceinline__ uint32_t bf16_pair(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// dst[i] = src[i] for n float4, every thread issuing up to kSepLd loads before its stores
__device__ __forceinline__ void sep_copy(float4* dst, const float4* src, int n) {
  for (int base = 0; base < n; base += kSepLd * 256) {
    float4 v[kSepLd];
#pragma unroll
    for (int k = 0; k < kSepLd; ++k) {
      const int i = base + k * 256 + (int)threadIdx.x;
      if (i < n) v[k] = __ldg(src + i);
    }
#pragma unroll
    for (int k = 0; k < kSepLd; ++k) {
      const int i = base + k * 256 + (int)threadIdx.x;
      if (i < n) dst[i] = v[k];
    }
  }
}

// global -> shared bulk copy (16-byte aligned addresses, a multiple of 16 bytes), completing
// `bytes` of transaction count on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// float2 entries of the S double buffer, which also stages Fz before the quads are formed
__host__ __device__ __forceinline__ int sep1_buf_elems(int n_el, int ny, int nx) {
  const int rows = 2 * kSepRows * nx * ny, stage = n_el * ny + 1;
  return ((rows > stage ? rows : stage) + 1) & ~1;
}

// FULL: n_el a multiple of 64 (every warp's elevations exist, no predicates).
template <bool FULL>
__global__ void __launch_bounds__(256, 2) k_sep1(Sep1Args a) {
  extern __shared__ float4 sep_smem[];
  const int nx = a.nx, ny = a.ny, M = nx * ny, nfz = a.n_el * ny;
  float4* fz4 = sep_smem;                                    // [n_el][ny]
  float2* buf = reinterpret_cast<float2*>(fz4 + nfz);        // [2][kSepRows][M]
  uint64_t* bars = reinterpret_cast<uint64_t*>(buf + sep1_buf_elems(a.n_el, ny, nx));
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // Fz as quads: (Re, Re, Im, Im) for the mirrored-row sums below, else (Re, Im, Im, Re)
  {
    float2* fzq = buf;  // staging: the S rows come later
    sep_copy(reinterpret_cast<float4*>(fzq), reinterpret_cast<const float4*>(a.fz), nfz / 2);
    if ((nfz & 1) && tid == 0) fzq[nfz - 1] = a.fz[nfz - 1];
    __syncthreads();
    for (int i = tid; i < nfz; i += blockDim.x) {
      const float2 f = fzq[i];
      fz4[i] = FULL ? make_float4(f.x, f.x, f.y, f.y) : make_float4(f.x, f.y, f.y, f.x);
    }
    fence_proxy_async();  // the staging accesses come before the copies' writes into the buffer
    __syncthreads();
  }
  pdl_wait();  // the element echoes come from the synthesis
  const int npairs = (a.nr + kSepRows - 1) / kSepRows, units = npairs * a.n_pings;
  // thread 0's count of copies issued into and received by each half of the buffer
  int issued0 = 0, issued1 = 0, landed0 = 0, landed1 = 0;
  auto issue = [&](int u, int b) {
    const int p = u / npairs, n0 = (u - p * npairs) * kSepRows;
    const uint32_t bytes = (uint32_t)(min(kSepRows, a.nr - n0) * M) * 8u;
    const uint32_t bar = smem_u32(&bars[b]);
    mbar_expect_tx(bar, bytes);
    bulk_g2s(smem_u32(buf + b * kSepRows * M), a.S + ((int64_t)p * a.nr_pad + kPad + n0) * M, bytes, bar);
    if (b) ++issued1; else ++issued0;
  };
  if (tid == 0 && (int)blockIdx.x < units) issue(blockIdx.x, 0);
  uint16_t* xh = reinterpret_cast<uint16_t*>(a.x_hi);
  uint16_t* xl = reinterpret_cast<uint16_t*>(a.x_lo);
  const int mxl = lane < nx ? lane : 0;  // lanes past nx compute on column 0 and write zeros
  int k = 0;
  for (int u = blockIdx.x; u < units; u += gridDim.x, ++k) {
    const int b = k & 1;
    if (tid == 0 && u + (int)gridDim.x < units) issue(u + gridDim.x, b ^ 1);
    const int p = u / npairs, n0 = (u - p * npairs) * kSepRows;
    const int rows = min(kSepRows, a.nr - n0);
    float2* srow = buf + b * kSepRows * M;
    // a ragged last unit: zero rows past the copy (bytes the copy does not write)
    if (rows < kSepRows) {
      for (int i = rows * M + tid; i < kSepRows * M; i += blockDim.x) srow[i] = make_float2(0.f, 0.f);
      fence_proxy_async();  // before a later copy into this half
    }
    const bool ok = mbar_wait(smem_u32(&bars[b]), (uint32_t)(k >> 1) & 1u, a.err);
    if (tid == 0 && ok) { if (b) ++landed1; else ++landed0; }
    if (__syncthreads_or(!ok)) break;
    auto put = [&](int el, int r, float2 v) {
      if (lane >= nx) v = make_float2(0.f, 0.f);
      const int64_t row = ((int64_t)el * a.n_pings + p) * a.nr_x + n0 + r;
      const int64_t off = row * a.k_pad + 2 * lane;  // 16-bit units
      const uint32_t hi = bf16_pair(v.x, v.y);
      *reinterpret_cast<uint32_t*>(xh + off) = hi;
      if (a.mode == SONAR_FP32) {
        __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&hi);
        const float2 hf = __bfloat1622float2(h);
        *reinterpret_cast<uint32_t*>(xl + off) = bf16_pair(v.x - hf.x, v.y - hf.y);
      }
    };
    if constexpr (FULL) {
      // Mirrored elevation rows: the cell-centred grid is symmetric, sin(el) of row
      // n_el - 1 - j is minus that of row j, so (the taper being real) Fz[n_el - 1 - j] =
      // conj Fz[j]. With A = sum_my Re Fz[j][my] s and B = sum_my Im Fz[j][my] s the two
      // rows' sums are A + jB and A - jB: half the multiply-adds, each a packed product of
      // a real weight with a complex sample. Warp w takes rows j = w + 8 i (i < 4) of every
      // 32 and their mirrors.
      const int half = a.n_el / 2;
      for (int j0 = w; j0 < half; j0 += 32) {
        float2 A0[4], B0[4], A1[4], B1[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) A0[i] = B0[i] = A1[i] = B1[i] = make_float2(0.f, 0.f);
        const float4* fzr = fz4 + j0 * ny;
#pragma unroll 8
        for (int my = 0; my < ny; ++my) {
          const float2 s0 = srow[my * nx + mxl], s1 = srow[M + my * nx + mxl];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float4 f = fzr[8 * i * ny + my];  // (Re, Re, Im, Im)
            A0[i] = __ffma2_rn(make_float2(f.x, f.y), s0, A0[i]);
            B0[i] = __ffma2_rn(make_float2(f.z, f.w), s0, B0[i]);
            A1[i] = __ffma2_rn(make_float2(f.x, f.y), s1, A1[i]);
            B1[i] = __ffma2_rn(make_float2(f.z, f.w), s1, B1[i]);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int j = j0 + 8 * i;
#pragma unroll
          for (int r = 0; r < kSepRows; ++r) {
            if (r >= rows) break;
            const float2 A = r == 0 ? A0[i] : A1[i], B = r == 0 ? B0[i] : B1[i];
            put(j, r, make_float2(A.x - B.y, A.y + B.x));
            put(a.n_el - 1 - j, r, make_float2(A.x + B.y, A.y - B.x));
          }
        }
      }
    } else {
      for (int e0 = w; e0 < a.n_el; e0 += 64) {
        float2 acc0[8], acc1[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc0[i] = acc1[i] = make_float2(0.f, 0.f);
        const float4* fzr = fz4 + e0 * ny;
#pragma unroll 4
        for (int my = 0; my < ny; ++my) {
          const float2 s0 = srow[my * nx + mxl], s1 = srow[M + my * nx + mxl];
          const float2 sx0 = make_float2(s0.x, s0.x), sy0 = make_float2(-s0.y, s0.y);
          const float2 sx1 = make_float2(s1.x, s1.x), sy1 = make_float2(-s1.y, s1.y);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (e0 + 8 * i < a.n_el) {
              // (re, im) += s f: (s.x f.x - s.y f.y, s.x f.y + s.y f.x)
              const float4 f = fzr[8 * i * ny + my];
              acc0[i] = __ffma2_rn(sy0, make_float2(f.z, f.w), __ffma2_rn(sx0, make_float2(f.x, f.y), acc0[i]));
              acc1[i] = __ffma2_rn(sy1, make_float2(f.z, f.w), __ffma2_rn(sx1, make_float2(f.x, f.y), acc1[i]));
            }
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int el = e0 + 8 * i;
          if (el >= a.n_el) continue;
#pragma unroll
          for (int r = 0; r < kSepRows; ++r) {
            if (r >= rows) break;
            put(el, r, r == 0 ? acc0[i] : acc1[i]);
          }
        }
      }
    }
    __syncthreads();  // this half is read out before the copy two units on refills it
  }
  // after a copy that never landed: wait (bounded) for this CTA's copies still in flight
  if (tid == 0) {
    if (issued0 > landed0) mbar_wait(smem_u32(&bars[0]), (uint32_t)landed0 & 1u, a.err);
    if (issued1 > landed1) mbar_wait(smem_u32(&bars[1]), (uint32_t)landed1 & 1u, a.err);
  }
}

// Fz quads, the S double buffer (also the Fz staging area), two mbarriers
size_t sep1_smem(int n_el, int ny, int nx) {
  return sizeof(float4) * n_el * ny + sizeof(float2) * sep1_buf_elems(n_el, ny, nx) + 2 * sizeof(uint64_t);
}

}  // namespace

cudaError_t launch_steer(const SteerArgs& a, cudaStream_t st) {
  k_steer<<<a.n_levels > 1 ? 8192 : 1024, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// Dynamic shared-memory opt-in of the GEMM kernels (once per device, outside capture),
// and for the cluster variants the number of clusters that fit on the device.
int g_mc_clusters[4][2][2];  // [tile 256, 224, 192, 128][one product, three][cluster 2, 4]
constexpr int tile_index(int bn) { return bn == 256 ? 0 : bn == 224 ? 1 : bn == 192 ? 2 : 3; }

template <int BN, int NPASS, int CS>
cudaLaunchConfig_t gemm_config(int grid, cudaStream_t st, cudaLaunchAttribute (&attr)[2]) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kGemmThreads);
  cfg.dynamicSmemBytes = gemm_smem<BN, NPASS>();
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = CS;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = CS > 1 ? 2 : 1;
  return cfg;
}

template <int BN, int NPASS, int CS>
cudaError_t gemm_attr_cs() {
  cudaError_t e = cudaFuncSetAttribute(k_gemm<BN, NPASS, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)gemm_smem<BN, NPASS>());
  if (e != cudaSuccess || CS == 1) return e;
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = gemm_config<BN, NPASS, CS>(CS, 0, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_gemm<BN, NPASS, CS>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;  // this cluster size is not used
  }
  g_mc_clusters[tile_index(BN)][NPASS == 3 ? 1 : 0][CS == 4 ? 1 : 0] = n;
  return cudaSuccess;
}
template <int BN, int NPASS>
cudaError_t gemm_attr_one() {
  cudaError_t e;
  if ((e = gemm_attr_cs<BN, NPASS, 1>()) != cudaSuccess) return e;
  if ((e = gemm_attr_cs<BN, NPASS, 2>()) != cudaSuccess) return e;
  return gemm_attr_cs<BN, NPASS, 4>();
}
template <int BN>
cudaError_t gemm_attr() {
  cudaError_t e = gemm_attr_one<BN, 1>();
  return e != cudaSuccess ? e : gemm_attr_one<BN, 3>();
}
bool sep1_supported(int nx, int ny) { return nx >= 1 && nx <= 32 && ny >= 1 && ny <= 64 && (nx * ny) % 2 == 0; }

cudaError_t launch_sep1(const Sep1Args& a, int sm_count, cudaStream_t st) {
  if (!sep1_supported(a.nx, a.ny) || a.n_el * a.ny > kSepMaxFz || a.k_pad != 64 || a.nr < 1 || a.n_pings < 1)
    return cudaErrorInvalidValue;
  const size_t smem = sep1_smem(a.n_el, a.ny, a.nx);
  const int units = (a.nr + kSepRows - 1) / kSepRows * a.n_pings;
  const dim3 grid((unsigned)(units < 2 * sm_count ? units : 2 * sm_count));
  cudaError_t e = a.n_el % 64 == 0 ? launch_pdl(k_sep1<true>, grid, dim3(256), smem, st, a)
                                   : launch_pdl(k_sep1<false>, grid, dim3(256), smem, st, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t prepare_gemm() {
  const int sep_max = (int)sep1_smem(kSepMaxFz / 64, 64, 32);  // the largest Fz and S rows
  cudaError_t e = cudaFuncSetAttribute(k_sep1<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sep_max);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sep1<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sep_max);
  if (e != cudaSuccess) return e;
  if ((e = gemm_attr<256>()) != cudaSuccess) return e;
  if ((e = gemm_attr<224>()) != cudaSuccess) return e;
  if ((e = gemm_attr<192>()) != cudaSuccess) return e;
  return gemm_attr<128>();
}

bool gemm_cluster_fits(int cs, int tiles_m, int tile_n, int n_phase) {
  if (cs == 1) return true;
  if ((cs != 2 && cs != 4) || tiles_m % cs != 0) return false;
  return g_mc_clusters[tile_index(tile_n)][n_phase == 3 ? 1 : 0][cs == 4 ? 1 : 0] > 0;
}

int gemm_cluster_size(int tiles_m, int tile_n, int n_phase, int sm_count) {
  (void)sm_count;
  // Measured on the C2 ping (N tile 224, bench stage events): the FP32 form 0.1147 /
  // 0.1106 / 0.1331 ms with 1 / 2 / 4 CTAs per cluster, the one-product form 0.0553 /
  // 0.0573 / 0.0676 ms. Four lose because every stage waits for the slowest of four CTAs
  // to release it; the one-product form, whose MMAs per stage are short, gains nothing
  // from sharing B once sixteen warps drain its tiles.
  if (n_phase != 3) return 1;
  const int* n = g_mc_clusters[tile_index(tile_n)][1];
  if (tiles_m % 2 == 0 && n[0] > 0) return 2;
  return 1;
}

template <int BN, int NPASS, int CS>
cudaError_t launch_cs(const GemmArgs& a, int sm_count, cudaStream_t st, uint32_t idesc) {
  const int n_tiles = a.tiles_m * a.tiles_n;
  int grid;
  if (CS > 1) {
    const int n_groups = n_tiles / CS, nc = g_mc_clusters[tile_index(BN)][NPASS == 3 ? 1 : 0][CS == 4 ? 1 : 0];
    grid = CS * (n_groups < nc ? n_groups : nc);
  } else {
    grid = n_tiles < sm_count ? n_tiles : sm_count;
  }
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = gemm_config<BN, NPASS, CS>(grid, st, attr);
  return cudaLaunchKernelEx(&cfg, k_gemm<BN, NPASS, CS>, a, idesc);
}

template <int BN, int NPASS>
cudaError_t launch_np(const GemmArgs& a, int sm_count, cudaStream_t st) {
  const uint32_t idesc = make_idesc(a.f16 ? 0 : 1, BM, BN);
  switch (a.cluster) {
    case 4: return launch_cs<BN, NPASS, 4>(a, sm_count, st, idesc);
    case 2: return launch_cs<BN, NPASS, 2>(a, sm_count, st, idesc);
    default: return launch_cs<BN, NPASS, 1>(a, sm_count, st, idesc);
  }
}

template <int BN>
cudaError_t launch_bn(const GemmArgs& a, int sm_count, cudaStream_t st) {
  return a.n_phase == 3 ? launch_np<BN, 3>(a, sm_count, st) : launch_np<BN, 1>(a, sm_count, st);
}

cudaError_t launch_gemm(const GemmArgs& a, int sm_count, cudaStream_t st) {
  if (a.cluster != 1 && a.cluster != 2 && a.cluster != 4) return cudaErrorInvalidValue;
  if (a.tiles_m % a.cluster != 0) return cudaErrorInvalidValue;
  if (a.cluster > 1 && g_mc_clusters[tile_index(a.tile_n)][a.n_phase == 3 ? 1 : 0][a.cluster == 4 ? 1 : 0] <= 0)
    return cudaErrorInvalidValue;
  cudaError_t e;
  switch (a.tile_n) {
    case 256: e = launch_bn<256>(a, sm_count, st); break;
    case 224: e = launch_bn<224>(a, sm_count, st); break;
    case 192: e = launch_bn<192>(a, sm_count, st); break;
    case 128: e = launch_bn<128>(a, sm_count, st); break;
    default: return cudaErrorInvalidValue;
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_peaks(const PeakArgs& a, cudaStream_t st) {
  const int nb = a.n_beam_az * a.n_beam_el;
  cudaError_t e = launch_pdl(k_peaks, dim3((unsigned)ceil_div(nb, 1024), a.n_pings), dim3(1024), 0, st, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sonar
