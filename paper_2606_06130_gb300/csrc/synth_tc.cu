// Element-echo synthesis on the 5th-generation tensor cores.
//
// Element phasors are separable, exp(j k_a u.p_m) = ey[mx] ez[my], so the echoes of a
// tile of T consecutive range samples are complex contractions over the hits k of
//   S[n][my nx + mx] = sum_k g_k(n) ey_k[mx] ez_k[my],   g_k(n) = c_k R(t_n - tau_k).
// Each hit contributes two K columns (re, im); the MMA shape is M = 128 and N = 64, 128
// or 192 (32, 64 or 96 complex output columns per tile).
//
// Persistent CTAs take equal contiguous ranges of the delay-sorted hits and walk them in
// K-blocks of up to 32 hits whose taps stay inside a few tiles. Generator warps form the
// operands in BF16 (the FP32 form also writes the residual lo parts and runs three
// passes hi*hi, hi*lo, lo*hi); one thread issues tcgen05.mma into a ring of TMEM
// accumulators, one per tile; four epilogue warps add a tile's accumulator into S (FP32,
// vector atomics) once the walk has passed it. N operands are stored as the real
// 4-form: a row (Re b, -Im b) gives the real part and a row (Im b, Re b) the imaginary
// part of each complex output.
//
// k_synth_tz (arrays of nx ny = 128 L2 elements): with my = my_hi L2 + my_lo the z
//   phasor factors as ez[my] = E1[my_hi] E2[my_lo] (E1 = ez at L2 my_hi, E2[my_lo] =
//   exp(j theta_z my_lo)). The M operand A[(my_hi, mx)][k] = ey[mx] E1[my_hi], one phase
//   per entry, does not depend on the tile: it is written once per K-block into tensor
//   memory (tcgen05.st), which the MMA reads as A. Only the N operand B[k][(re/im, n,
//   my_lo)] = g_k(n) E2[my_lo] (T = NP / L2 samples for NP complex columns) is formed per
//   tile, in shared memory. Every MMA costs a fixed issue time whatever its N, so wider
//   tiles (NP = 64, 96) need fewer of them; the price is fewer TMEM accumulators
//   (384 / 2 NP) and so fewer tiles per K-block. The sixteen generator warps form four
//   independent groups, one per MMA K step (8 hits), each with one warp per TMEM lane
//   quarter and its own named barrier. The pulse autocorrelation is real (even window,
//   chirp centred on t = 0), so B = R_k(n) (c_k E2[my_lo]) with R_k(n) real: c_k joins the
//   per-hit E2 factor (L2 complex products per hit) and each B entry is one packed FP32
//   product R (Re, -Im) of c_k E2. A fifth warp per group (the stage helper) works one
//   K-block ahead: it moves the records and forms the taps and the c_k E2 factors, so
//   the four operand warps only form A and B. One walker warp walks the K-blocks for
//   everyone but the epilogue: it feeds the helpers' descriptor ring, and group 0's
//   helper forwards each descriptor to the MMA issuer.
// k_synth_tc (small arrays): A[(n, mx)][k] = g_k(n) ey[mx] per tile (T = 128 / nx) and
//   B[k][(my, re/im)] = ez[my] once per K-block, both in shared memory.
#include <limits.h>
#include <stddef.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace sonar {
namespace {
using namespace tc;

constexpr int KH = 32;           // hits per K-block: K = 64 BF16 columns (re, im)
constexpr int TMAX = 5;          // tiles one K-block may touch (k_synth_tc)
constexpr int kGenWarps = 16;
constexpr int kGenWarp0 = 5;     // warp 0: MMA, warps 1..4: epilogue, warps 5..20: generators
                                 // (k_synth_tz: operand warps, then the stage helpers)
constexpr int kThreadsTC = 32 * (kGenWarp0 + kGenWarps);
constexpr int kGenThreads = 32 * kGenWarps;
constexpr int M_BYTES = 128 * 128;  // 128 rows x 64 BF16
constexpr int N_BYTES = 64 * 128;   // 64 rows x 64 BF16
constexpr int kMaxAx = 64;

// k_synth_tc rings
constexpr int NA = 3;            // per-tile A slots (hi + lo)
constexpr int NB = 2;            // per-K-block B slots (hi + lo)
constexpr int RING = 8;          // TMEM accumulators of 64 columns
// k_synth_tz
constexpr int kGroups = 4;
constexpr int KG = KH / kGroups;   // hits per generator group = one MMA K step
constexpr int kAcol = 384;         // TMEM columns of the two per-K-block A slots (hi 32, lo 32)
// Stage helpers: warps 21..24 for groups 0..3 (one per SM sub-partition, warp w runs on
// w % 4), then the walker, warp 25. Each stage helper is a latency-bound chain that its
// group's barrier waits on. While each helper still walked the K-blocks itself, the one
// sharing sub-partition 0 with the MMA issuer (whose tcgen05.mma issue stalls that
// sub-partition for much of every K-block) made its group about 1250 cycles late per
// K-block; with the walk moved to the walker, the helpers keep up on every
// sub-partition (measured: 0.157 ms for this layout, 0.160 ms with the walker on
// sub-partition 0 and two helpers on sub-partition 1).
constexpr int kHelper0 = kGenWarp0 + kGenWarps;  // 21
constexpr int kWalkerWarp = kHelper0 + 4;        // 25, sub-partition 1
constexpr int kHelper3 = kHelper0 + 3;           // 24, sub-partition 0
constexpr int kThreadsTZ = 32 * (kHelper0 + kGroups + 1);  // 832
constexpr int kWRing = 16;                       // walker -> helpers descriptor ring
constexpr int kGroupThreads = 32 * 5;                   // four operand warps and the helper

// Tile shape of k_synth_tz for NP complex output columns per tile.
template <int NP>
struct ZShape {
  static constexpr int N_ROWS = 2 * NP;               // B rows = MMA N: NP real, NP imaginary
  static constexpr int B_BYTES = N_ROWS * 128;        // one 128-byte swizzled row per B row
  static constexpr int RING = kAcol / N_ROWS;         // TMEM accumulators below the A slots
  static constexpr int NT = NP == 32 ? 8 : (NP == 64 ? 4 : 3);  // per-tile B slots (hi + lo)
  static constexpr int TMAXZ = RING < 5 ? RING : 5;   // tiles one K-block may touch
};

// The walk over tiles that every role repeats identically. Tiles are numbered by a
// virtual index that only grows; an epoch maps tile base + i to the rows origin + T i ..
// origin + T i + T - 1. A K-block may open a new epoch at its first row (origin = that row,
// base past every tile used so far), which retires all live tiles.
struct TileWalk {
  int origin = -1, base = 0;           // current epoch (origin < 0: none yet)
  int live_lo = INT_MAX, live_hi = -1;  // tiles that may still receive MMAs
  __device__ __forceinline__ int row0(int t, int T) const { return origin + (t - base) * T; }
};
// Rows per tile T = MUL 2^s. Every quotient the walk takes is of a non-negative row
// offset, so floor division by T is a shift and a division by the compile-time MUL (a
// multiply-high), off the MMA issuer's critical path.
template <int MUL>
struct TileRows {
  int s;
  __device__ __forceinline__ int T() const { return MUL << s; }
  __device__ __forceinline__ int div(int x) const { return (int)((unsigned)(x >> s) / (unsigned)MUL); }
};
struct KBlk {
  int cnt, t_first, t_last;
  int origin, base;  // the epoch this K-block uses
};

// First-tap rows of the 32 sorted hits from h (lane i holds hit h + i; INT_MAX past the
// end). Loaded one K-block ahead so the latency overlaps the current K-block's work.
__device__ __forceinline__ int load_window(const int32_t* ng, int64_t h, int64_t h_end, int lane) {
  const int64_t idx = h + lane;
  return idx < h_end ? __ldg(&ng[idx]) : INT_MAX;
}

// K-block starting at the window's first hit: as many hits (<= 32) as keep every tap
// inside tmax tiles of T rows from the K-block's first tile. It stays in the current
// epoch unless a new epoch at its first row n0 covers its hits with fewer tiles per hit
// (an epoch at n0 needs ceil((span + W) / T) tiles, the fixed grid up to one more).
// Warp-cooperative (all 32 lanes), identical in every role. Rows are sorted and
// non-negative, so n0 >= origin and the integer quotients are floor divisions.
template <int MUL>
__device__ __forceinline__ KBlk kblock_from(int v, const TileRows<MUL>& tr, int tmax, int W, const TileWalk& w) {
  const int T = tr.T();
  const int n0 = __shfl_sync(0xffffffffu, v, 0);
  int tf = 0, tl = 0, cnt = 0;
  if (w.origin >= 0) {
    tf = tr.div(n0 - w.origin);
    const int lim = w.origin + (tf + tmax) * T - W;
    cnt = __popc(__ballot_sync(0xffffffffu, v <= lim));
    if (cnt < 1) cnt = 1;  // cannot happen for W <= T (tmax - 1) + 1
    tl = tr.div(__shfl_sync(0xffffffffu, v, cnt - 1) + W - 1 - w.origin);
  }
  const int lim_f = n0 + tmax * T - W;
  int cnt_f = __popc(__ballot_sync(0xffffffffu, v <= lim_f));
  if (cnt_f < 1) cnt_f = 1;
  const int tl_f = tr.div(__shfl_sync(0xffffffffu, v, cnt_f - 1) + W - 1 - n0);
  KBlk k;
  if (w.origin < 0 || (tl_f + 1) * cnt < (tl - tf + 1) * cnt_f) {
    k.origin = n0;
    k.base = w.live_hi + 1;
    k.cnt = cnt_f;
    k.t_first = k.base;
    k.t_last = k.base + tl_f;
  } else {
    k.origin = w.origin;
    k.base = w.base;
    k.cnt = cnt;
    k.t_first = w.base + tf;
    k.t_last = w.base + tl;
  }
  return k;
}
__device__ __forceinline__ void walk_advance(TileWalk& w, const KBlk& kb) {
  w.origin = kb.origin;
  w.base = kb.base;
  w.live_lo = kb.t_first;
  if (kb.t_last > w.live_hi) w.live_hi = kb.t_last;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_lo(float a, float b, uint32_t hi) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&hi);
  float2 f = __bfloat1622float2(h);
  return pack_bf16(a - f.x, b - f.y);
}
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void sts64(uint32_t addr, uint32_t a, uint32_t b) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void red_add2(float* dst, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(dst), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void named_bar(uint32_t id, uint32_t n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ float2 cmul(float2 p, float2 q) {
  return make_float2(p.x * q.x - p.y * q.y, p.x * q.y + p.y * q.x);
}

// One 16-byte operand chunk (4 complex values, hits 4c..4c+3) in the 128-byte swizzle.
__device__ __forceinline__ void store_chunk(uint32_t hi_base, uint32_t lo_base, int row, int c, const float2 (&v)[4],
                                            bool fp32_form) {
  uint32_t hv[4], lv[4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    hv[kk] = pack_bf16(v[kk].x, v[kk].y);
    lv[kk] = pack_lo(v[kk].x, v[kk].y, hv[kk]);
  }
  const uint32_t off = (uint32_t)(row * 128 + ((c ^ (row & 7)) << 4));
  sts128(hi_base + off, hv[0], hv[1], hv[2], hv[3]);
  if (fp32_form) sts128(lo_base + off, lv[0], lv[1], lv[2], lv[3]);
}

// sin(pi x), cos(pi x) for the element phasors, which only feed BF16 operands (2^-9
// rounding, 2^-17 with the hi/lo split): x is reduced exactly to r in [-1, 1]
// (x - 2 rint(x / 2) has no rounding for |x| < 2^22), then the hardware sine and cosine
// on [-pi, pi] (absolute error ~5e-7).
__device__ __forceinline__ void sincospi_operand(float x, float* s, float* c) {
  const float r = x - 2.0f * rintf(0.5f * x);
  __sincosf(3.14159265358979f * r, s, c);
}

// Tap c_k R(u) from the shared-memory pulse table by 4-point Lagrange interpolation
// (error ~4e-8); zero outside the pulse support.
__device__ __forceinline__ float2 tap_value(const float2* tab, float scale, float u, float cr, float ci) {
  float2 g = make_float2(0.f, 0.f);
  const float x = u * scale + (float)(kRTabS / 2 + 2);
  if (x >= 1.0f && x < (float)(kRTabS + 3)) {
    const int i = (int)x;
    const float f = x - (float)i;
    const float wm = -f * (f - 1.f) * (f - 2.f) * (1.f / 6.f);
    const float w0 = (f + 1.f) * (f - 1.f) * (f - 2.f) * 0.5f;
    const float w1 = -(f + 1.f) * f * (f - 2.f) * 0.5f;
    const float w2 = (f + 1.f) * f * (f - 1.f) * (1.f / 6.f);
    const float2 r0 = tab[i - 1], r1 = tab[i], r2 = tab[i + 1], r3 = tab[i + 2];
    const float rr = wm * r0.x + w0 * r1.x + w1 * r2.x + w2 * r3.x;
    const float ri = wm * r0.y + w0 * r1.y + w1 * r2.y + w2 * r3.y;
    g = make_float2(cr * rr - ci * ri, cr * ri + ci * rr);
  }
  return g;
}

// Real tap R(u) from the real part of the shared-memory pulse table (4-point Lagrange,
// zero outside the pulse support). The autocorrelation of the Hann-windowed chirp centred
// on t = 0 is real: R(u) = (1/E) int w(s + u/2) w(s - u/2) exp(j 2 pi kappa u s) ds with
// the window product even in s, so only the cosine part survives (the table's imaginary
// parts are rounding noise of the closed form).
__device__ __forceinline__ float tap_real(const float* tab, float scale, float u) {
  float g = 0.f;
  const float x = u * scale + (float)(kRTabS / 2 + 2);
  if (x >= 1.0f && x < (float)(kRTabS + 3)) {
    const int i = (int)x;
    const float f = x - (float)i;
    const float wm = -f * (f - 1.f) * (f - 2.f) * (1.f / 6.f);
    const float w0 = (f + 1.f) * (f - 1.f) * (f - 2.f) * 0.5f;
    const float w1 = -(f + 1.f) * f * (f - 2.f) * 0.5f;
    const float w2 = (f + 1.f) * f * (f - 1.f) * (1.f / 6.f);
    g = fmaf(wm, tab[i - 1], fmaf(w0, tab[i], fmaf(w1, tab[i + 1], w2 * tab[i + 2])));
  }
  return g;
}

// Residual lo = bf16(v - hi) of a pair packed as hi = (bf16(v.x), bf16(v.y)); the
// difference is exact in FP32 (Sterbenz), one packed FP32 operation for both halves.
__device__ __forceinline__ uint32_t pack_lo2(float2 v, uint32_t hi) {
  const float2 hf = make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u));
  const float2 d = __ffma2_rn(hf, make_float2(-1.f, -1.f), v);
  return pack_bf16(d.x, d.y);
}

#define TMEM_LD_16(taddr, r)                                                                               \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), \
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),         \
                 "=r"(r[15])                                                                                   \
               : "r"(taddr))

#define TMEM_LD_8(taddr, r)                                                                       \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"                 \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]) \
               : "r"(taddr))

// Bounded wait that gives up for good once any role of the CTA has timed out.
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
  if (*abort_flag) return false;
  if (mbar_wait(bar, parity, err)) return true;
  *abort_flag = 1;
  return false;
}

// Epilogue role (warps 1..4): walks the K-blocks like the MMA issuer and, for every tile
// the walk has passed, adds the accumulator columns of its TMEM slot into S. dst(u, pr)
// is the S entry of complex column pr of this thread's lane row in tile u; the real and
// imaginary parts sit in adjacent columns (2 pr, 2 pr + 1) of a 64-column accumulator,
// or, with HALVES, in columns pr and NP + pr of a 2 NP-column one. R accumulators, at
// most tmax tiles per K-block, T rows per tile.
template <int R, bool HALVES, int NP, class TR, class Dst>
__device__ __forceinline__ void epilogue_role(const SynthArgs& a, int64_t h0, int64_t h1, TR tr, int tmax, int W,
                                              int q, int lane, uint32_t tmem_base, uint64_t* tdone,
                                              uint64_t* tfree, volatile int* abort_flag, int n_cols, Dst dst) {
  constexpr int SLOT_COLS = HALVES ? 2 * NP : 64;
  uint32_t par = 0, cur = 0;  // per slot: parity of its use count, parity of the tile it holds
  TileWalk w;
  auto flush = [&](int u) {
    const int64_t r0 = w.row0(u, tr.T());
    const int slot = u % R;
    const bool ok = wait_or_abort(smem_u32(&tdone[slot]), (cur >> slot) & 1u, abort_flag, a.err);
    if (ok) {
      tc_fence_after();
      const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(slot * SLOT_COLS);
      if (HALVES) {
        for (int c0 = 0; c0 < NP; c0 += 8) {
          uint32_t re[8], im[8];
          TMEM_LD_8(ta + c0, re);
          TMEM_LD_8(ta + NP + c0, im);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int i = 0; i < 8; ++i) red_add2(dst(r0, c0 + i), __uint_as_float(re[i]), __uint_as_float(im[i]));
        }
      } else {
        for (int c0 = 0; c0 < n_cols; c0 += 16) {
          uint32_t v[16];
          TMEM_LD_16(ta + c0, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int i = 0; i < 8; ++i) red_add2(dst(r0, c0 / 2 + i), __uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
        }
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&tfree[slot]));
  };
  int win = load_window(a.sorted_n, h0, h1, lane);
  for (int64_t h = h0; h < h1;) {
    const KBlk kb = kblock_from(win, tr, tmax, W, w);
    const int64_t hn = h + kb.cnt;
    win = load_window(a.sorted_n, hn, h1, lane);
    for (int u = w.live_lo; u <= w.live_hi && u < kb.t_first; ++u) flush(u);  // in their own epoch
    for (int t = (w.live_hi + 1 > kb.t_first ? w.live_hi + 1 : kb.t_first); t <= kb.t_last; ++t) {
      const uint32_t bit = 1u << (t % R);
      cur = (cur & ~bit) | (par & bit);
      par ^= bit;
    }
    walk_advance(w, kb);
    h = hn;
  }
  for (int u = w.live_lo; u <= w.live_hi; ++u) flush(u);
}

__device__ __forceinline__ void tmem_alloc_512(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(512)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free_512(uint32_t base) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(512) : "memory");
}

// =====================================================================================
// k_synth_tz: z-split operands, per-K-block A in tensor memory
// =====================================================================================
// Records are stored into the stage as 16-byte vectors: every stage starts on a 16-byte
// boundary (alignas makes the size a multiple of 16 too).
// Stage buffers per generator group, used round robin by K-block. Three, so that the one
// a K-block's records are written into (during the previous K-block, before the group's
// barrier) was last read two K-blocks earlier: every warp of the group has passed the
// intervening barrier since, including the A-operand reads that follow a K-block's own
// barrier. With two, a fast warp could overwrite records a slow one was still reading.
// The K-block's walk descriptor travels with its records (written by the group's walker
// warp one K-block ahead).
constexpr int kZStages = 3;
template <int WT>
struct alignas(16) ZStage {  // one generator group's 8 hits of one K-block
  HitRec rec[KG];
  int n[KG];
  int kb[8];               // cnt, t_first, t_last, origin, base of the K-block
  float4 g[WT + 1][KG];    // taps R as (Re, Re, Im, Im), tap-major; row WT stays zero
  float2 e2[KG][32];       // (Re, -Im) of c_k E2[my_lo], my_lo < L2 <= 32
};

static_assert(sizeof(ZStage<8>) % 16 == 0 && sizeof(ZStage<12>) % 16 == 0 && sizeof(ZStage<16>) % 16 == 0,
              "stages hold 16-byte vector stores");
static_assert(offsetof(ZStage<8>, rec) % 16 == 0, "records are 16-byte aligned in a stage");

template <int WT, int NP>
constexpr size_t tz_smem_bytes() {
  using Z = ZShape<NP>;
  return 1024 + (size_t)Z::NT * 2 * Z::B_BYTES + kZStages * kGroups * sizeof(ZStage<WT>) + 64 * 8 + 64;
}

// CT: complex taps (the raw series' pulse table); otherwise the taps are real (the pulse
// autocorrelation) and each B entry is one packed FP32 product.
template <int WT, int NP, bool CT>
__global__ void __launch_bounds__(kThreadsTZ, 1) k_synth_tz(SynthArgs a, uint32_t idesc) {
  using Z = ZShape<NP>;
  constexpr int NT = Z::NT, RING = Z::RING, B_BYTES = Z::B_BYTES;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // align by pointer arithmetic on the shared array, so that the compiler keeps the
  // shared address space (an integer round trip would turn every access generic)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sB = smem;  // NT x (hi, lo) per-tile N operands
  ZStage<WT>(*zst)[kGroups] = reinterpret_cast<ZStage<WT>(*)[kGroups]>(sB + NT * 2 * B_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(&zst[kZStages][0]);
  uint64_t* tb_full = bars;
  uint64_t* tb_empty = bars + NT;
  uint64_t* am_full = bars + 2 * NT;
  uint64_t* am_empty = am_full + 2;
  uint64_t* tdone = am_empty + 2;
  uint64_t* tfree = tdone + RING;
  uint64_t* done = tfree + RING;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  __shared__ float s_rre[CT ? 1 : kRTabS + 5];    // real pulse autocorrelation
  __shared__ float2 s_rtab[CT ? kRTabS + 5 : 1];  // complex pulse (raw series)
  __shared__ int4 s_mkd[8][2];                     // K-block descriptors for the MMA issuer
  __shared__ int4 s_wkd[kWRing][2];                // K-block descriptors for the stage helpers
  __shared__ uint64_t s_wfull[kWRing], s_wempty[kWRing];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = a.nx, ny = a.ny, M = nx * ny;
  const int L2 = M / 128, lL2 = 31 - __clz(L2);  // my_lo count, a power of two
  const int lnx = 31 - __clz(nx);                 // nx is a power of two
  const TileRows<NP / 32> tr{5 - lL2};           // T = NP / L2 rows per tile
  const int T = tr.T();
  const int W = a.taps;
  const bool fp32_form = a.n_pass == 3;

  for (int i = threadIdx.x; i < kRTabS + 5; i += blockDim.x) {
    if constexpr (CT) s_rtab[i] = a.rtab_s[i];
    else s_rre[i] = a.rtab_s[i].x;
  }
  for (int i = threadIdx.x; i < kZStages * kGroups * KG; i += blockDim.x)
    zst[i / (kGroups * KG)][(i / KG) % kGroups].g[WT][i % KG] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NT; ++i) {
      mbar_init(smem_u32(&tb_full[i]), kGenWarps);
      mbar_init(smem_u32(&tb_empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) { mbar_init(smem_u32(&am_full[i]), kGenWarps); mbar_init(smem_u32(&am_empty[i]), 1); }
    for (int i = 0; i < RING; ++i) { mbar_init(smem_u32(&tdone[i]), 1); mbar_init(smem_u32(&tfree[i]), 4); }
    mbar_init(smem_u32(done), 1);
    for (int i = 0; i < kWRing; ++i) {
      mbar_init(smem_u32(&s_wfull[i]), 1);
      mbar_init(smem_u32(&s_wempty[i]), kGroups);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc_512(tmem_slot);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // the hits come from the binning kernels
  pdl_wait();
  // this CTA's range of the sorted hits: cost-balanced by the binning scan, else equal
  const int64_t Hn = *a.n_valid;
  const int64_t h0 = a.bounds ? (int64_t)a.bounds[blockIdx.x] : Hn * blockIdx.x / gridDim.x;
  const int64_t h1 = a.bounds ? (int64_t)a.bounds[blockIdx.x + 1] : Hn * (blockIdx.x + 1) / gridDim.x;

  if (warp == 0) {
    // ------------------------------------------------------------- MMA issuer
    // One thread. It does not walk the K-blocks itself: each K-block's descriptor comes
    // from the ring s_mkd, written by group 0's stage helper before the group barrier
    // that precedes the A signal it waits for (a walk here, a latency-bound chain on a
    // busy sub-partition, left the tensor pipe idle between K-blocks). Slot j & 7 is
    // rewritten for K-block j + 8, after group 0 has formed A of K-block j + 6, which
    // waited for this thread's release of K-block j + 4.
    if (lane == 0) {
      uint32_t used = 0, par = 0;  // per slot: held a tile before, parity of its use count
      TileWalk w;
      int j = 0;
      unsigned tix = 0;
      for (int64_t h = h0; h < h1;) {
        const int aslot = j & 1;
        if (!wait_or_abort(smem_u32(&am_full[aslot]), (j >> 1) & 1, abort_flag, a.err)) break;
        const int4 d0 = s_mkd[j & 7][0];
        KBlk kb;
        kb.cnt = d0.x;
        kb.t_first = d0.y;
        kb.t_last = d0.z;
        kb.origin = d0.w;
        kb.base = s_mkd[j & 7][1].x;
        // tiles the walk has passed: their accumulators are final once these MMAs land
        for (int u = w.live_lo; u <= w.live_hi && u < kb.t_first; ++u) tc_commit(smem_u32(&tdone[u % RING]));
        const uint32_t ah = tmem_base + (uint32_t)(kAcol + aslot * 64), al = ah + 32;
        for (int t = kb.t_first; t <= kb.t_last; ++t) {
          const int slot = t % RING;
          const bool fresh = t > w.live_hi;
          bool ok = true;
          if (fresh) {
            const uint32_t bit = 1u << slot;
            if (used & bit) ok = wait_or_abort(smem_u32(&tfree[slot]), ((par >> slot) & 1u) ^ 1u, abort_flag, a.err);
            used |= bit;
            par ^= bit;
          }
          const int bslot = (int)(tix % NT);
          ok = ok && wait_or_abort(smem_u32(&tb_full[bslot]), (tix / NT) & 1, abort_flag, a.err);
          if (ok) {
            tc_fence_after();
            const uint32_t d = tmem_base + (uint32_t)(slot * Z::N_ROWS);
            // K step kk advances B by 32 bytes: +2 in the descriptor's address field
            const uint64_t bdh = sw128_desc(smem_u32(sB + bslot * 2 * B_BYTES));
            const uint64_t bdl = bdh + (B_BYTES >> 4);
            tc_mma4_tmem_a(d, ah, bdh, idesc, fresh ? 0u : 1u);
            if (fp32_form) {
              tc_mma4_tmem_a(d, ah, bdl, idesc, 1u);
              tc_mma4_tmem_a(d, al, bdh, idesc, 1u);
            }
            tc_commit(smem_u32(&tb_empty[bslot]));
          }
          ++tix;
        }
        tc_commit(smem_u32(&am_empty[aslot]));
        walk_advance(w, kb);
        ++j;
        h += kb.cnt;
      }
      for (int u = w.live_lo; u <= w.live_hi; ++u) tc_commit(smem_u32(&tdone[u % RING]));
      tc_commit(smem_u32(done));
      mbar_wait(smem_u32(done), 0, a.err);
      // executed tensor work: per tile issue n_pass x 4 MMAs of M 128, N 2 NP, K 16
      if (a.mma_flop) atomicAdd(a.mma_flop, (unsigned long long)tix * a.n_pass * 4ull * (2ull * 128 * 2 * NP * 16));
    }
    __syncwarp();
  } else if (warp < kGenWarp0) {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int L = q * 32 + lane;
    const int my_hi = L >> lnx, mx = L & (nx - 1);
    epilogue_role<RING, true, NP>(a, h0, h1, tr, Z::TMAXZ, W, q, lane, tmem_base, tdone, tfree, abort_flag, 2 * NP,
                                  [&](int64_t r0, int pr) {
                                    const int nl = pr >> lL2, my_lo = pr & (L2 - 1);
                                    const int64_t row = r0 + nl;
                                    return reinterpret_cast<float*>(a.S + row * M + (my_hi * L2 + my_lo) * nx + mx);
                                  });
  } else if (warp == kWalkerWarp) {
    // ------------------------------------------------------------- walker
    // Walks the K-blocks (the walk every role used to repeat) and hands each descriptor
    // to the four stage helpers through a ring of kWRing slots: slot s is refilled once
    // all four have taken it. Its first-tap windows are loaded one K-block ahead.
    TileWalk w;
    int j = 0;
    int win = load_window(a.sorted_n, h0, h1, lane);
    for (int64_t h = h0; h < h1; ++j) {
      const KBlk k = kblock_from(win, tr, Z::TMAXZ, W, w);
      walk_advance(w, k);
      win = load_window(a.sorted_n, h + k.cnt, h1, lane);
      const int slot = j % kWRing;
      if (!wait_or_abort(smem_u32(&s_wempty[slot]), ((j / kWRing) & 1) ^ 1, abort_flag, a.err)) break;
      if (lane == 0) {
        s_wkd[slot][0] = make_int4(k.cnt, k.t_first, k.t_last, k.origin);
        s_wkd[slot][1] = make_int4(k.base, 0, 0, 0);
        mbar_arrive(smem_u32(&s_wfull[slot]));
      }
      __syncwarp();
      h += k.cnt;
    }
  } else if (warp >= kHelper0) {
    // ------------------------------------------------------------- stage helpers
    // One warp per generator group works one K-block ahead of the group's four operand
    // warps: it takes the walker's descriptors, moves the records (fetched two K-blocks
    // ahead, so the loads overlap a whole K-block) and forms the taps R and the factors
    // c_k E2 into the stage the operand warps take next. The group's named barrier at the
    // top of every K-block hands one stage over; the stage written after barrier j is the
    // one the operand warps last read during K-block j - 2, before barrier j - 1.
    const int grp = warp == kHelper3 ? kGroups - 1 : warp - kHelper0;
    const uint32_t bar_id = 1 + grp;
    const float pl2 = 2.0f * a.pitch_over_lambda;
    // lanes 0-15 move the group's 8 records (hit lane / 2, half lane & 1)
    auto fetch = [&](int64_t hs) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      const int64_t k = hs + KG * grp + (lane >> 1);
      if (lane < 2 * KG && k < h1) v = __ldg(reinterpret_cast<const uint4*>(a.hits_sorted + k) + (lane & 1));
      return v;
    };
    auto put_rec = [&](ZStage<WT>& S, uint4 v) {
      if (lane < 2 * KG) reinterpret_cast<uint4*>(&S.rec[lane >> 1])[lane & 1] = v;
      __syncwarp();  // the records are read back by other lanes below
    };
    // the descriptor and the first-tap rows (padding hits: INT_MIN / 2) of a filled stage
    auto put_kb = [&](ZStage<WT>& S, const KBlk& k, int jk) {
      if (lane == 0) *reinterpret_cast<int4*>(S.kb) = make_int4(k.cnt, k.t_first, k.t_last, k.origin);
      if (lane == 1) S.kb[4] = k.base;
      if (grp == 0 && lane == 2) s_mkd[jk & 7][0] = make_int4(k.cnt, k.t_first, k.t_last, k.origin);
      if (grp == 0 && lane == 3) s_mkd[jk & 7][1] = make_int4(k.base, 0, 0, 0);
      if (lane < KG) S.n[lane] = lane < k.cnt - KG * grp ? S.rec[lane].nglob : INT_MIN / 2;
    };
    auto fill = [&](ZStage<WT>& S) {
      // taps R((u0 + i) dt) (c_k rides in the E2 factor). A padding hit's first row is
      // INT_MIN / 2, so every tap index of it reads the zero row WT: its taps are formed
      // like the others' (no dependence on the walk) and never read.
#pragma unroll
      for (int it = 0; it < (KG * WT + 31) / 32; ++it) {
        const int item = lane + 32 * it;
        if (item < KG * WT) {
          const int kl = item & (KG - 1), qq = item >> 3;
          float2 g = make_float2(0.f, 0.f);
          if (qq < W) {
            const float u0 = S.rec[kl].u0 + (float)qq;
            if constexpr (CT) g = tap_value(s_rtab, a.rtab_s_scale, u0, 1.f, 0.f);
            else g.x = tap_real(s_rre, a.rtab_s_scale, u0);
          }
          S.g[qq][kl] = make_float4(g.x, g.x, g.y, g.y);
        }
      }
      // (Re, -Im) of c_k E2[my_lo], E2[my_lo] = exp(j 2 pi (d/lambda) my_lo u_z)
#pragma unroll 2
      for (int item = lane; item < KG * L2; item += 32) {
        const int kl = item & (KG - 1), ql = item >> 3;
        const float4 r = *reinterpret_cast<const float4*>(&S.rec[kl]);  // nglob, u0, cr, ci
        float s, c;
        sincospi_operand(pl2 * (float)ql * S.rec[kl].uz, &s, &c);
        S.e2[kl][ql] = make_float2(fmaf(r.z, c, -r.w * s), -fmaf(r.z, s, r.w * c));
      }
    };
    // descriptor jk from the walker's ring; after an abort (the walker gave up) a K-block
    // of 32 hits in the last tile, so that every role still runs out its K-blocks in step
    KBlk kc{};
    auto get_kb = [&](int jk) {
      const int slot = jk % kWRing;
      KBlk k = kc;
      k.cnt = KH;
      k.t_first = k.t_last = kc.t_last;
      if (wait_or_abort(smem_u32(&s_wfull[slot]), (jk / kWRing) & 1, abort_flag, a.err)) {
        const int4 d0 = s_wkd[slot][0];
        k.cnt = d0.x;
        k.t_first = d0.y;
        k.t_last = d0.z;
        k.origin = d0.w;
        k.base = s_wkd[slot][1].x;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&s_wempty[slot]));
      return k;
    };
    uint4 rec_ahead = make_uint4(0u, 0u, 0u, 0u);
    if (h0 < h1) {
      const uint4 r0 = fetch(h0);
      kc = get_kb(0);
      rec_ahead = fetch(h0 + kc.cnt);
      put_rec(zst[0][grp], r0);
      fill(zst[0][grp]);
      put_kb(zst[0][grp], kc, 0);
    }
    int j = 0;
    for (int64_t h = h0; h < h1;) {
      named_bar(bar_id, kGroupThreads);
      const int64_t hn = h + kc.cnt;
      if (hn < h1) {
        ZStage<WT>& Sn = zst[(j + 1) % kZStages][grp];
        put_rec(Sn, rec_ahead);
        const KBlk kn = get_kb(j + 1);
        rec_ahead = fetch(hn + kn.cnt);
        fill(Sn);
        put_kb(Sn, kn, j + 1);
        kc = kn;
      }
      ++j;
      h = hn;
    }
  } else {
    // ------------------------------------------------------------- operand warps
    const int gw = warp - kGenWarp0;
    const int grp = gw >> 2;            // hits KG grp .. KG grp + 7 of every K-block
    const int wi = gw & 3;              // warp in group
    const int q = warp & 3;             // TMEM lane quarter of this warp
    const uint32_t bar_id = 1 + grp;
    const float pl2 = 2.0f * a.pitch_over_lambda;
    // A operand: this thread's TMEM lane is row (my_hi, mx), element (mx, L2 my_hi)
    const int arow = q * 32 + lane, a_hi = arow >> lnx, a_mx = arow & (nx - 1);
    const float ax = pl2 * ((float)a_mx - 0.5f * (float)(nx - 1));
    const float az = pl2 * ((float)(L2 * a_hi) - 0.5f * (float)(ny - 1));
    // B operand: the group's share of a tile is NP complex columns pr = (n, my_lo) by its
    // 8 hits, written as rows pr (re) and NP + pr (im). A thread owns column c0 + 32 r (r <
    // NP / 32) and hit pair pp (hits 2 pp, 2 pp + 1: one 8-byte half of a 16-byte chunk),
    // so every thread has the same number of items per tile and keeps its hit pair, my_lo
    // and the column's swizzle phase for the whole kernel. Lanes 0-7 and 8-15 (one
    // half-warp, which an 8-byte store serves together) take eight consecutive columns at
    // one hit pair each: their 16-byte chunks (2 grp + pp / 2) ^ (c0 & 7) are all distinct,
    // so the half-warp's 128 bytes cover the 32 banks once.
    const int tg = wi * 32 + lane;
    const int pp = (tg & 31) >> 3, c0 = ((tg >> 5) << 3) | (tg & 7);  // column c0 + 32 r
    const int my_lo = c0 & (L2 - 1);
    const int nl0 = c0 >> lL2, nl_r = 32 >> lL2;          // tile row of column c0 + 32 r
    const uint32_t boff0 = (uint32_t)(c0 * 128 + (((2 * grp + (pp >> 1)) ^ (c0 & 7)) << 4) + ((pp & 1) << 3));
    int j = 0;
    unsigned tix = 0;
    for (int64_t h = h0; h < h1;) {
      // the helper has filled this K-block's stage
      named_bar(bar_id, kGroupThreads);
      ZStage<WT>& S = zst[j % kZStages][grp];
      const int4 kd = *reinterpret_cast<const int4*>(S.kb);
      KBlk kb;
      kb.cnt = kd.x;
      kb.t_first = kd.y;
      kb.t_last = kd.z;
      kb.origin = kd.w;
      kb.base = S.kb[4];
      const int64_t hn = h + kb.cnt;

      // per-K-block A operand: row (my_hi, mx) = this thread's TMEM lane, 8 columns
      const int aslot = j & 1;
      auto a_form = [&]() {
        wait_or_abort(smem_u32(&am_empty[aslot]), ((j >> 1) & 1) ^ 1, abort_flag, a.err);
        tc_fence_after();
        // ey[mx] E1[my_hi] = exp(j pi x), x = 2 (d/lambda) ((mx - (nx-1)/2) u_y + (L2 my_hi
        // - (ny-1)/2) u_z), reduced exactly to [-1, 1]. Padding hits (zero B rows) keep
        // finite entries: their records are zeros or real hits.
        uint32_t hi[KG], lo[KG];
#pragma unroll
        for (int kl = 0; kl < KG; kl += 2) {
          const float2 u0 = *reinterpret_cast<const float2*>(&S.rec[kl].uy);
          const float2 u1 = *reinterpret_cast<const float2*>(&S.rec[kl + 1].uy);
          const float2 x = make_float2(fmaf(ax, u0.x, az * u0.y), fmaf(ax, u1.x, az * u1.y));
          const float2 hx = __fmul2_rn(x, make_float2(0.5f, 0.5f));
          const float2 r = __ffma2_rn(make_float2(rintf(hx.x), rintf(hx.y)), make_float2(-2.f, -2.f), x);
          const float2 y = __fmul2_rn(r, make_float2(3.14159265358979f, 3.14159265358979f));
          float2 p0, p1;
          __sincosf(y.x, &p0.y, &p0.x);
          __sincosf(y.y, &p1.y, &p1.x);
          hi[kl] = pack_bf16(p0.x, p0.y);
          hi[kl + 1] = pack_bf16(p1.x, p1.y);
          lo[kl] = pack_lo2(p0, hi[kl]);
          lo[kl + 1] = pack_lo2(p1, hi[kl + 1]);
        }
        const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(kAcol + aslot * 64 + KG * grp);
        tmem_st8(ta, hi);
        if (fp32_form) tmem_st8(ta + 32, lo);
      };
      auto a_signal = [&]() {
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&am_full[aslot]));
      };

      // per-tile B operand: every generator thread writes NP / 32 items of every tile
      const int k0 = 2 * pp, k1 = k0 + 1;
      const int nk0 = S.n[k0], nk1 = S.n[k1];
      const float2 ea0 = S.e2[k0][my_lo], ea1 = S.e2[k1][my_lo];
      const float2 eb0 = make_float2(ea0.y, -ea0.x), eb1 = make_float2(ea1.y, -ea1.x);  // (-Im, -Re)
      const int ntiles = kb.t_last - kb.t_first + 1;
      const int row_first = kb.origin + (kb.t_first - kb.base) * T;  // first row of the first tile
      auto b_form = [&](int i) {
        const unsigned tqi = tix + (unsigned)i;
        const int bslot = (int)(tqi % NT);
        wait_or_abort(smem_u32(&tb_empty[bslot]), ((tqi / NT) & 1) ^ 1, abort_flag, a.err);
        const uint32_t bh = smem_u32(sB + bslot * 2 * B_BYTES), bl = bh + B_BYTES;
        const int trow0 = row_first + i * T + nl0;
#pragma unroll
        for (int r = 0; r < NP / 32; ++r) {
          const int trow = trow0 + r * nl_r;
          const uint32_t boff = boff0 + (uint32_t)(r * 32 * 128);
          // row pr: (Re b, -Im b) = g (Re E2, -Im E2) with the tap g real; row NP + pr:
          // (Im b, Re b) = the same BF16 pair with its halves swapped and the new low half
          // negated (rounding is sign-symmetric)
          float2 v0 = make_float2(0.f, 0.f), v1 = v0;
          const int tap0 = trow - nk0, tap1 = trow - nk1;
          if constexpr (CT) {
            // complex tap g: (Re b, -Im b) = Re g (Re E2, -Im E2) + Im g (-Im E2, -Re E2)
            if ((unsigned)tap0 < (unsigned)WT) {
              const float4 g = S.g[tap0][k0];
              v0 = __ffma2_rn(make_float2(g.z, g.w), eb0, __fmul2_rn(make_float2(g.x, g.y), ea0));
            }
            if ((unsigned)tap1 < (unsigned)WT) {
              const float4 g = S.g[tap1][k1];
              v1 = __ffma2_rn(make_float2(g.z, g.w), eb1, __fmul2_rn(make_float2(g.x, g.y), ea1));
            }
          } else {
            // taps outside 0 .. WT - 1 (and padding hits) read the zero row WT
            const unsigned c0i = min((unsigned)tap0, (unsigned)WT), c1i = min((unsigned)tap1, (unsigned)WT);
            v0 = __fmul2_rn(*reinterpret_cast<const float2*>(&S.g[c0i][k0]), ea0);
            v1 = __fmul2_rn(*reinterpret_cast<const float2*>(&S.g[c1i][k1]), ea1);
          }
          const uint32_t h0 = pack_bf16(v0.x, v0.y), h1 = pack_bf16(v1.x, v1.y);
          sts64(bh + boff, h0, h1);
          sts64(bh + boff + NP * 128, __byte_perm(h0, 0u, 0x1032) ^ 0x8000u, __byte_perm(h1, 0u, 0x1032) ^ 0x8000u);
          if (fp32_form) {
            const uint32_t l0 = pack_lo2(v0, h0), l1 = pack_lo2(v1, h1);
            sts64(bl + boff, l0, l1);
            sts64(bl + boff + NP * 128, __byte_perm(l0, 0u, 0x1032) ^ 0x8000u, __byte_perm(l1, 0u, 0x1032) ^ 0x8000u);
          }
        }
        return bslot;
      };
      auto b_signal = [&](int bslot) {
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tb_full[bslot]));
      };
      // the A operand's tensor-memory stores drain while the first tile's B entries are
      // formed; then both are signalled
      a_form();
      const int s0 = b_form(0);
      a_signal();
      b_signal(s0);
      for (int i = 1; i < ntiles; ++i) b_signal(b_form(i));
      tix += (unsigned)ntiles;
      ++j;
      h = hn;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_free_512(tmem_base);
  }
}

// =====================================================================================
// k_synth_tc: per-tile A = taps x ey, per-K-block B = ez (small arrays)
// =====================================================================================
template <int WT>
struct alignas(16) Stage {
  HitRec rec[KH];
  int n[KH];
  float2 g[WT][KH];        // tap-major: staging writes and operand reads are conflict-free
  float2 ey[KH][kMaxAx];   // per hit, element-major: a warp reads consecutive elements
  float2 ez[KH][kMaxAx];
};

static_assert(sizeof(Stage<8>) % 16 == 0 && sizeof(Stage<12>) % 16 == 0 && sizeof(Stage<16>) % 16 == 0,
              "stages hold 16-byte vector stores");

template <int WT>
constexpr size_t tc_smem_bytes() {
  return 1024 + (size_t)NA * 2 * M_BYTES + (size_t)NB * 2 * N_BYTES + 2 * sizeof(Stage<WT>) + 64 * 8 + 64;
}

__device__ __forceinline__ void gen_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kGenThreads) : "memory"); }

template <int WT>
__global__ void __launch_bounds__(kThreadsTC, 1) k_synth_tc(SynthArgs a, uint32_t idesc) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sA = smem;                          // per-tile A: NA x (hi, lo)
  uint8_t* sB = sA + NA * 2 * M_BYTES;         // per-K-block B: NB x (hi, lo)
  Stage<WT>* st = reinterpret_cast<Stage<WT>*>(sB + NB * 2 * N_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(st + 2);
  uint64_t* a_full = bars;
  uint64_t* a_empty = bars + NA;
  uint64_t* b_full = bars + 2 * NA;
  uint64_t* b_empty = bars + 2 * NA + NB;
  uint64_t* tdone = bars + 2 * NA + 2 * NB;
  uint64_t* tfree = tdone + RING;
  uint64_t* done = tfree + RING;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  __shared__ float2 s_rtab[kRTabS + 5];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = a.nx, ny = a.ny, M = nx * ny;
  const int lnx = 31 - __clz(nx);
  const TileRows<1> tr{7 - lnx};  // T = 128 / nx rows per tile
  const int T = tr.T();
  const int W = a.taps;
  const int n_cols = 2 * ny;
  const bool fp32_form = a.n_pass == 3;

  for (int i = threadIdx.x; i < kRTabS + 5; i += blockDim.x) s_rtab[i] = a.rtab_s[i];
  if (threadIdx.x == 0) {
    for (int i = 0; i < NA; ++i) { mbar_init(smem_u32(&a_full[i]), kGenWarps); mbar_init(smem_u32(&a_empty[i]), 1); }
    for (int i = 0; i < NB; ++i) { mbar_init(smem_u32(&b_full[i]), kGenWarps); mbar_init(smem_u32(&b_empty[i]), 1); }
    for (int i = 0; i < RING; ++i) { mbar_init(smem_u32(&tdone[i]), 1); mbar_init(smem_u32(&tfree[i]), 4); }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc_512(tmem_slot);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_wait();
  // this CTA's range of the sorted hits: cost-balanced by the binning scan, else equal
  const int64_t Hn = *a.n_valid;
  const int64_t h0 = a.bounds ? (int64_t)a.bounds[blockIdx.x] : Hn * blockIdx.x / gridDim.x;
  const int64_t h1 = a.bounds ? (int64_t)a.bounds[blockIdx.x + 1] : Hn * (blockIdx.x + 1) / gridDim.x;

  if (warp == 0) {
    // ------------------------------------------------------------- MMA issuer
    uint32_t used = 0, par = 0;
    TileWalk w;
    int j = 0, a_idx = 0;
    int win = load_window(a.sorted_n, h0, h1, lane);
    for (int64_t h = h0; h < h1;) {
      const KBlk kb = kblock_from(win, tr, TMAX, W, w);
      const int64_t hn = h + kb.cnt;
      win = load_window(a.sorted_n, hn, h1, lane);
      if (lane == 0) {
        for (int u = w.live_lo; u <= w.live_hi && u < kb.t_first; ++u) tc_commit(smem_u32(&tdone[u % RING]));
        const int bslot = j % NB;
        const bool b_ok = wait_or_abort(smem_u32(&b_full[bslot]), (j / NB) & 1, abort_flag, a.err);
        for (int t = kb.t_first; t <= kb.t_last; ++t) {
          const int slot = t % RING;
          const bool fresh = t > w.live_hi;
          bool ok = b_ok;
          if (fresh) {
            const uint32_t bit = 1u << slot;
            if (used & bit) ok = ok && wait_or_abort(smem_u32(&tfree[slot]), ((par >> slot) & 1u) ^ 1u, abort_flag, a.err);
            used |= bit;
            par ^= bit;
          }
          const int aslot = a_idx % NA;
          ok = ok && wait_or_abort(smem_u32(&a_full[aslot]), (a_idx / NA) & 1, abort_flag, a.err);
          if (ok) {
            tc_fence_after();
            const uint32_t d = tmem_base + (uint32_t)(slot * 64);
            const uint32_t ah = smem_u32(sA + aslot * 2 * M_BYTES), al = ah + M_BYTES;
            const uint32_t bh = smem_u32(sB + bslot * 2 * N_BYTES), bl = bh + N_BYTES;
            for (int pass = 0; pass < a.n_pass; ++pass) {
              const uint32_t aa = pass == 2 ? al : ah, bb = pass == 1 ? bl : bh;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                tc_mma(d, sw128_desc(aa + kk * 32), sw128_desc(bb + kk * 32), idesc,
                       (fresh && pass == 0 && kk == 0) ? 0u : 1u);
            }
            tc_commit(smem_u32(&a_empty[aslot]));
          }
          ++a_idx;
        }
        if (b_ok) tc_commit(smem_u32(&b_empty[bslot]));
      }
      walk_advance(w, kb);
      ++j;
      h = hn;
      __syncwarp();
    }
    if (lane == 0) {
      for (int u = w.live_lo; u <= w.live_hi; ++u) tc_commit(smem_u32(&tdone[u % RING]));
      tc_commit(smem_u32(done));
      mbar_wait(smem_u32(done), 0, a.err);
    }
    __syncwarp();
  } else if (warp < kGenWarp0) {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;
    const int L = q * 32 + lane;
    const int nl = L >> lnx, mx = L & (nx - 1);
    epilogue_role<RING, false, 32>(a, h0, h1, tr, TMAX, W, q, lane, tmem_base, tdone, tfree, abort_flag, n_cols, [&](int64_t r0, int my) {
      const int64_t row = r0 + nl;
      return reinterpret_cast<float*>(a.S + row * M + my * nx + mx);
    });
  } else {
    // ------------------------------------------------------------- operand generators
    const int gt = threadIdx.x - kGenWarp0 * 32;
    const float pl2 = 2.0f * a.pitch_over_lambda;
    int j = 0, a_idx = 0;
    // hit records are fetched one K-block ahead: 32 records from the K-block's first hit
    auto fetch_recs = [&](int64_t hs) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      const int64_t k = hs + (gt >> 1);
      if (gt < 2 * KH && k < h1) v = __ldg(reinterpret_cast<const uint4*>(a.hits_sorted + k) + (gt & 1));
      return v;
    };
    int win = load_window(a.sorted_n, h0, h1, lane);
    uint4 recv = fetch_recs(h0);
    TileWalk w;
    for (int64_t h = h0; h < h1;) {
      const KBlk kb = kblock_from(win, tr, TMAX, W, w);
      walk_advance(w, kb);
      const int64_t hn = h + kb.cnt;
      win = load_window(a.sorted_n, hn, h1, lane);
      Stage<WT>& S = st[j & 1];
      if (gt < 2 * KH) reinterpret_cast<uint4*>(&S.rec[gt >> 1])[gt & 1] = recv;
      recv = fetch_recs(hn);
      gen_bar();
      for (int item = gt; item < KH * WT; item += kGenThreads) {
        const int k = item & (KH - 1), qq = item >> 5;
        const bool valid = k < kb.cnt;
        const HitRec& hr = S.rec[k];
        float2 g = make_float2(0.f, 0.f);
        if (valid && qq < W) g = tap_value(s_rtab, a.rtab_s_scale, hr.u0 + (float)qq, hr.cr, hr.ci);
        S.g[qq][k] = g;
        if (qq == 0) S.n[k] = valid ? hr.nglob : INT_MIN / 2;
      }
      for (int item = gt; item < KH * nx; item += kGenThreads) {
        const int mx = item & (nx - 1), k = item >> lnx;
        float2 e = make_float2(0.f, 0.f);
        if (k < kb.cnt) {
          float s, c;
          sincospi_operand(pl2 * ((float)mx - 0.5f * (float)(nx - 1)) * S.rec[k].uy, &s, &c);
          e = make_float2(c, s);
        }
        S.ey[k][mx] = e;
      }
      for (int item = gt; item < KH * ny; item += kGenThreads) {
        const int k = item / ny, my = item - k * ny;
        float2 e = make_float2(0.f, 0.f);
        if (k < kb.cnt) {
          float s, c;
          sincospi_operand(pl2 * ((float)my - 0.5f * (float)(ny - 1)) * S.rec[k].uz, &s, &c);
          e = make_float2(c, s);
        }
        S.ez[k][my] = e;
      }
      gen_bar();
      // per-K-block B[k][(my, re/im)] = 4-form of ez[my]
      const int bslot = j % NB;
      wait_or_abort(smem_u32(&b_empty[bslot]), ((j / NB) & 1) ^ 1, abort_flag, a.err);
      {
        const uint32_t bh = smem_u32(sB + bslot * 2 * N_BYTES), bl = bh + N_BYTES;
        for (int idx = gt; idx < n_cols * 8; idx += kGenThreads) {
          const int c = idx / n_cols, row = idx - c * n_cols;
          const int my = row >> 1, r = row & 1;
          float2 v[4];
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const float2 e = S.ez[4 * c + kk][my];
            v[kk] = r == 0 ? make_float2(e.x, -e.y) : make_float2(e.y, e.x);
          }
          store_chunk(bh, bl, row, c, v, fp32_form);
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&b_full[bslot]));
      // per-tile A[(n, mx)][k] = g_k(n) ey[mx]; a warp covers 32 rows of one chunk
      for (int t = kb.t_first; t <= kb.t_last; ++t) {
        const int aslot = a_idx % NA;
        wait_or_abort(smem_u32(&a_empty[aslot]), ((a_idx / NA) & 1) ^ 1, abort_flag, a.err);
        const uint32_t ah = smem_u32(sA + aslot * 2 * M_BYTES), al = ah + M_BYTES;
        for (int idx = gt; idx < 128 * 8; idx += kGenThreads) {
          const int c = idx >> 7, row = idx & 127;
          const int nl = row >> lnx, mx = row & (nx - 1);
          const int trow = kb.origin + (t - kb.base) * T + nl;
          float2 v[4];
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const int k = 4 * c + kk;
            const int tap = trow - S.n[k];
            v[kk] = (tap >= 0 && tap < WT) ? cmul(S.g[tap][k], S.ey[k][mx]) : make_float2(0.f, 0.f);
          }
          store_chunk(ah, al, row, c, v, fp32_form);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&a_full[aslot]));
        ++a_idx;
      }
      ++j;
      h = hn;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_free_512(tmem_base);
  }
}

bool z_split(int nx, int ny) {
  const int M = nx * ny;
  if (M % 128 != 0) return false;
  const int L2 = M / 128;
  return L2 <= 32 && (32 % L2) == 0 && ny % L2 == 0 && nx >= 4 && nx <= kMaxAx && (nx & (nx - 1)) == 0 &&
         nx * (ny / L2) == 128 && ny / L2 + L2 <= kMaxAx;
}

// Shared memory per CTA: dynamic bytes plus the static pulse table (4136 bytes, padded
// to the 1024-byte alignment of the dynamic array), within the 227 KB a CTA may hold.
static_assert(tz_smem_bytes<16, 96>() + 7 * 1024 <= 227 * 1024, "z-split tile fits");
static_assert(tc_smem_bytes<16>() + 5 * 1024 <= 227 * 1024, "per-tile kernel fits");

// A z-split tile of NP complex columns holds T = NP / L2 whole rows, and a K-block of
// tap span W must fit in TMAXZ of them.
template <int NP>
bool zs_fits(int nx, int ny, int W) {
  const int L2 = nx * ny / 128;
  return NP % L2 == 0 && W <= (NP / L2) * (ZShape<NP>::TMAXZ - 1) + 1;
}

// Complex columns per z-split tile (0: no z-split shape applies). want (32, 64, 96) is
// taken when it fits; otherwise 96, then 64, then 32. An MMA costs about the same issue
// time whatever its N, so 96 columns need a third of the MMAs of 32; and with T = 12
// rows an 11-tap K-block of one row fits one tile, which also halves the B operand rows
// formed per K-block against 64 columns. Measured on 32x32 arrays (1024-bin ping, 534k
// hits), 64 / 96 columns: FP32 form 0.248 / 0.225 ms, BF16 0.215 / 0.205 ms; 32 columns
// took 30% longer than 64 (FP32 form).
int zs_pairs(int nx, int ny, int W, int want) {
  if (!z_split(nx, ny)) return 0;
  const bool f32 = zs_fits<32>(nx, ny, W), f64 = zs_fits<64>(nx, ny, W), f96 = zs_fits<96>(nx, ny, W);
  if ((want == 32 && f32) || (want == 64 && f64) || (want == 96 && f96)) return want;
  return f96 ? 96 : (f64 ? 64 : (f32 ? 32 : 0));
}

template <int WT, bool CT>
cudaError_t set_attr_tz() {
  cudaError_t e = cudaFuncSetAttribute(k_synth_tz<WT, 32, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tz_smem_bytes<WT, 32>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_synth_tz<WT, 64, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tz_smem_bytes<WT, 64>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_synth_tz<WT, 96, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tz_smem_bytes<WT, 96>());
  return e;
}

template <int WT>
cudaError_t set_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_synth_tc<WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes<WT>());
  if (e == cudaSuccess) e = set_attr_tz<WT, false>();
  if (e == cudaSuccess) e = set_attr_tz<WT, true>();
  return e;
}

template <int WT, bool CT>
cudaError_t launch_tz(const SynthArgs& a, int zs_np, int sm_count, cudaStream_t st) {
  if (zs_np == 32)
    return launch_pdl(k_synth_tz<WT, 32, CT>, dim3(sm_count), dim3(kThreadsTZ), tz_smem_bytes<WT, 32>(), st, a,
                      make_idesc(1, 128, 64));
  if (zs_np == 64)
    return launch_pdl(k_synth_tz<WT, 64, CT>, dim3(sm_count), dim3(kThreadsTZ), tz_smem_bytes<WT, 64>(), st, a,
                      make_idesc(1, 128, 128));
  return launch_pdl(k_synth_tz<WT, 96, CT>, dim3(sm_count), dim3(kThreadsTZ), tz_smem_bytes<WT, 96>(), st, a,
                    make_idesc(1, 128, 192));
}

template <int WT>
cudaError_t launch_one(const SynthArgs& a, int zs_np, int sm_count, cudaStream_t st) {
  if (zs_np == 32 || zs_np == 64 || zs_np == 96)
    return a.cplx_taps ? launch_tz<WT, true>(a, zs_np, sm_count, st) : launch_tz<WT, false>(a, zs_np, sm_count, st);
  return launch_pdl(k_synth_tc<WT>, dim3(sm_count), dim3(kThreadsTC), tc_smem_bytes<WT>(), st, a,
                    make_idesc(1, 128, 2 * a.ny));
}

}  // namespace

bool synth_tz_applies(int nx, int ny, int taps) { return taps <= 16 && zs_pairs(nx, ny, taps, 0) != 0; }

bool synth_tc_supported(int nx, int ny, int taps) {
  if (taps > 16) return false;
  if (z_split(nx, ny)) return zs_pairs(nx, ny, taps, 0) != 0;
  const bool pow2 = nx >= 4 && nx <= 64 && (nx & (nx - 1)) == 0;
  return pow2 && ny % 8 == 0 && ny >= 8 && ny <= 32 && taps <= (128 / nx) * (TMAX - 1) + 1;
}

cudaError_t prepare_synth_tc() {
  cudaError_t e;
  if ((e = set_attr<8>()) != cudaSuccess) return e;
  if ((e = set_attr<12>()) != cudaSuccess) return e;
  return set_attr<16>();
}

cudaError_t launch_synth_tc(const SynthArgs& a, int want_pairs, int sm_count, cudaStream_t st) {
  const int zs_np = zs_pairs(a.nx, a.ny, a.taps, want_pairs);
  cudaError_t e;
  if (a.taps <= 8) e = launch_one<8>(a, zs_np, sm_count, st);
  else if (a.taps <= 12) e = launch_one<12>(a, zs_np, sm_count, st);
  else e = launch_one<16>(a, zs_np, sm_count, st);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace sonar
