// Delay binning and element-echo synthesis (Sec. II.B: complex baseband accumulated per
// element with the phase set by the delay; echoes are formed already pulse-compressed,
// i.e. each hit contributes c_k R(t_n - tau_k) to the samples inside its pulse window).
//
// Binning is a counting sort of hits by the global index of their first tap. The
// synthesis runs persistent CTAs over equal chunks of the sorted hit list; a thread
// owns four elements and keeps a sliding window of `taps` samples in registers, so the
// inner loop is 4 FMAs per (hit, element, tap). Finished samples are flushed with
// vector atomics into S [rows][M] (FP32 complex), rows padded per ping.
#include "common.cuh"

namespace sonar {
namespace {

// Exclusive scan of counts (single CTA of 1024 threads); offsets[n_bins] = total.
// With `bounds`, it also splits the sorted hits into G ranges of equal estimated
// synthesis cost, one per persistent synthesis CTA: a hit costs 1 and every non-empty
// row `beta` more (sparse rows cut K-blocks short and spread them over more tiles, so a
// hit costs more there than in a dense row). bounds[0] = 0, bounds[G] = total; within a
// row the row's extra cost comes first.
__global__ void __launch_bounds__(1024) k_scan(const int32_t* counts, int32_t n_bins, int32_t* offsets, int32_t* cursor,
                                               int32_t* bounds, int G, int beta) {
  __shared__ int32_t wsum[32], wne[32], tot[2];
  pdl_wait();
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int per = (n_bins + 1023) / 1024;
  const int b0 = t * per, b1 = min(b0 + per, n_bins);
  int32_t s = 0, ne = 0;
  for (int b = b0; b < b1; ++b) {
    const int32_t c = counts[b];
    s += c;
    ne += c > 0;
  }
  // inclusive scans of (hits, non-empty rows): within each warp by shuffles, then of the
  // 32 warp totals by one warp
  int32_t xs = s, xn = ne;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t ys = __shfl_up_sync(0xffffffffu, xs, o), yn = __shfl_up_sync(0xffffffffu, xn, o);
    if (lane >= o) { xs += ys; xn += yn; }
  }
  if (lane == 31) { wsum[wid] = xs; wne[wid] = xn; }
  __syncthreads();
  if (wid == 0) {
    int32_t vs = wsum[lane], vn = wne[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t ys = __shfl_up_sync(0xffffffffu, vs, o), yn = __shfl_up_sync(0xffffffffu, vn, o);
      if (lane >= o) { vs += ys; vn += yn; }
    }
    wsum[lane] = vs - wsum[lane];  // exclusive prefix of the warp totals
    wne[lane] = vn - wne[lane];
    if (lane == 31) { tot[0] = vs; tot[1] = vn; }
  }
  __syncthreads();
  int32_t run = wsum[wid] + xs - s, nrun = wne[wid] + xn - ne;
  const int32_t total = tot[0];
  const int64_t C = (int64_t)total + (int64_t)beta * tot[1];  // total cost
  if (bounds && C == 0)
    for (int k = t; k <= G; k += 1024) bounds[k] = 0;
  for (int b = b0; b < b1; ++b) {
    const int32_t cnt = counts[b];  // counts and cursor may alias
    offsets[b] = run;
    cursor[b] = run;
    if (bounds && cnt > 0 && C > 0) {
      // boundaries k with lo <= k C / G < hi fall in this row's cost interval [lo, hi)
      const int64_t lo = (int64_t)run + (int64_t)beta * nrun, hi = lo + cnt + beta;
      for (int64_t k = (lo * G + C - 1) / C; k < G && k * C < hi * G; ++k) {
        if (k < 1) continue;
        const int64_t num = k * C - (lo + beta) * G;  // cost past the row's extra, times G
        int64_t j = num <= 0 ? 0 : (num + G - 1) / G;
        if (j > cnt) j = cnt;
        bounds[k] = run + (int32_t)j;
      }
    }
    run += cnt;
    nrun += cnt > 0;
  }
  if (t == 1023) {
    offsets[n_bins] = total;
    if (bounds) {
      bounds[0] = 0;
      bounds[G] = total;
    }
  }
}

// Each hit carries its rank among its row's hits (from the histogram atomic at emission),
// so it moves to offsets[row] + rank with no atomics. Records move as two 16-byte vectors.
__global__ void k_scatter(const HitRec* hits, const unsigned long long* n_hits, int32_t n_bins,
                          const int32_t* offsets, const int32_t* rank, HitRec* sorted, int32_t* sorted_n) {
  pdl_wait();
  const int64_t n = (int64_t)*n_hits;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  static_assert(sizeof(HitRec) == 32, "HitRec is two 16-byte vectors");
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4* src = reinterpret_cast<const uint4*>(hits + i);
    const uint4 v0 = __ldg(src), v1 = __ldg(src + 1);
    const int g = (int)v0.x;  // nglob is the record's first word
    if (g < 0 || g >= n_bins) continue;
    const int pos = __ldg(&offsets[g]) + __ldg(&rank[i]);
    uint4* dst = reinterpret_cast<uint4*>(sorted + pos);
    dst[0] = v0;
    dst[1] = v1;
    sorted_n[pos] = g;
  }
}

constexpr int kSub = 32;        // hits staged per round
constexpr int kThreads = 256;   // 4 elements per thread -> 1024 elements per CTA
constexpr int kMaxAxis = 64;    // nx, ny <= 64

__device__ __forceinline__ void red_add4(float* dst, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

template <int WT>
__global__ void __launch_bounds__(kThreads, 1) k_synth(SynthArgs a, const int32_t* total_ptr) {
  __shared__ int s_n[kSub];
  __shared__ float2 s_g[kSub][WT];
  __shared__ float2 s_ey[kSub][kMaxAxis];
  __shared__ float2 s_ez[kSub][kMaxAxis];
  pdl_wait();

  const int nx = a.nx, ny = a.ny, M = nx * ny;
  const int64_t H = *total_ptr;
  const int n_eb = (M + 4 * kThreads - 1) / (4 * kThreads);
  // equal chunks, about four work items per resident CTA
  int64_t target = (int64_t)gridDim.x * 4;
  int64_t chunk = ((H * n_eb + target - 1) / target + kSub - 1) / kSub * kSub;
  if (chunk < kSub) chunk = kSub;
  if (chunk > 8192) chunk = 8192;
  const int64_t n_chunks = (H + chunk - 1) / chunk;
  const int64_t n_items = n_chunks * n_eb;
  const int tid = threadIdx.x;

  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int64_t c = item / n_eb;
    const int eb = (int)(item % n_eb);
    const int m0 = eb * 4 * kThreads + 4 * tid;
    const bool active = m0 < M;
    const int mx0 = active ? m0 % nx : 0, my = active ? m0 / nx : 0;
    const int64_t h0 = c * chunk, h1 = min(h0 + chunk, H);
    float2 acc[WT][4];
#pragma unroll
    for (int i = 0; i < WT; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][e] = make_float2(0.f, 0.f);
    int base = -1;
    float2* S = a.S;

    auto flush_row = [&](int row) {
      if (active) {
        float* dst = reinterpret_cast<float*>(S + (int64_t)row * M + m0);
        red_add4(dst, acc[0][0].x, acc[0][0].y, acc[0][1].x, acc[0][1].y);
        red_add4(dst + 4, acc[0][2].x, acc[0][2].y, acc[0][3].x, acc[0][3].y);
      }
    };

    for (int64_t s0 = h0; s0 < h1; s0 += kSub) {
      const int nsub = (int)(h1 - s0 < kSub ? h1 - s0 : kSub);
      __syncthreads();
      // stage taps c_k R((u0 + i) dt) and the separable element phasors of each hit
      const int per_hit = WT + nx + ny;
      for (int idx = tid; idx < nsub * per_hit; idx += kThreads) {
        const int k = idx / per_hit, j = idx % per_hit;
        const HitRec& h = a.hits_sorted[s0 + k];
        if (j == 0) s_n[k] = h.nglob;
        if (j < WT) {
          float2 g = make_float2(0.f, 0.f);
          if (j < a.taps) {
            float x = (h.u0 + (float)j) * a.rtab_scale + (float)(kRTab / 2);
            if (x >= 0.f && x < (float)kRTab) {
              int i0 = (int)x;
              float f = x - (float)i0;
              float2 r0 = __ldg(&a.rtab[i0]), r1 = __ldg(&a.rtab[i0 + 1]);
              float rr = r0.x + f * (r1.x - r0.x), ri = r0.y + f * (r1.y - r0.y);
              g = make_float2(h.cr * rr - h.ci * ri, h.cr * ri + h.ci * rr);
            }
          }
          s_g[k][j] = g;
        } else if (j < WT + nx) {
          const int q = j - WT;
          float s, cc;
          sincospif(2.0f * a.pitch_over_lambda * ((float)q - 0.5f * (float)(nx - 1)) * h.uy, &s, &cc);
          s_ey[k][q] = make_float2(cc, s);
        } else {
          const int q = j - WT - nx;
          float s, cc;
          sincospif(2.0f * a.pitch_over_lambda * ((float)q - 0.5f * (float)(ny - 1)) * h.uz, &s, &cc);
          s_ez[k][q] = make_float2(cc, s);
        }
      }
      __syncthreads();
      for (int k = 0; k < nsub; ++k) {
        const int g = s_n[k];
        if (base < 0) base = g;
        if (g - base >= WT) {
#pragma unroll
          for (int i = 0; i < WT; ++i) {
            flush_row(base);
#pragma unroll
            for (int r = 0; r < WT - 1; ++r)
#pragma unroll
              for (int e = 0; e < 4; ++e) acc[r][e] = acc[r + 1][e];
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[WT - 1][e] = make_float2(0.f, 0.f);
            ++base;
          }
          base = g;
        }
        while (base < g) {
          flush_row(base);
#pragma unroll
          for (int r = 0; r < WT - 1; ++r)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[r][e] = acc[r + 1][e];
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[WT - 1][e] = make_float2(0.f, 0.f);
          ++base;
        }
        const float2 ez = s_ez[k][my];
        float2 E[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 ey = s_ey[k][mx0 + e];
          E[e] = make_float2(ey.x * ez.x - ey.y * ez.y, ey.x * ez.y + ey.y * ez.x);
        }
#pragma unroll
        for (int i = 0; i < WT; ++i) {
          const float2 gi = s_g[k][i];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            acc[i][e].x = fmaf(gi.x, E[e].x, fmaf(-gi.y, E[e].y, acc[i][e].x));
            acc[i][e].y = fmaf(gi.x, E[e].y, fmaf(gi.y, E[e].x, acc[i][e].y));
          }
        }
      }
    }
    if (base >= 0) {
#pragma unroll
      for (int i = 0; i < WT; ++i) {
        flush_row(base);
#pragma unroll
        for (int r = 0; r < WT - 1; ++r)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[r][e] = acc[r + 1][e];
        ++base;
      }
    }
  }
}

// ----------------------------------------------------------------- wideband synthesis
// Element echoes with the plane-wave delay across the aperture in the envelope as well
// as in the phase (the input of true-time-delay beamforming), at one of U phases per work
// item. A thread owns one element and a window of WT rows from e1 rows before each hit's
// first tap row; per (hit, element) it forms the phasor c_k ey[mx] ez[my] and the table
// position of the window's first row, x0 = x_hit + dy[mx] + dz[my] (the element's delay
// in table entries), then reads row i at entry floor(x0) + i U F with the one weight
// x0 - floor(x0): 8 instructions per (hit, element, row). The table is zero outside the
// pulse support, so rows of the window the element's pulse does not reach add zero.
// Element order: an 8-lane quarter-warp (which a 16-byte shared load serves together)
// reads the table at its elements' delays, so its elements are kept close in delay: for
// 32-wide arrays each quarter-warp takes a block of 2 columns x 4 rows of elements (the
// vertical pitch weighs less: |u_z| <= sin(vfov / 2) is below |u_y|), which puts fewer
// of its eight addresses in the same bank group than eight elements along a row.
constexpr int kWbThreads = 256;  // one element per thread -> 256 elements per work item

// Element of thread t in work item eb: blocks of 2 x 4 per quarter-warp for nx = 32 (an
// item is 32 columns x 8 rows), the natural order otherwise.
__device__ __forceinline__ int wb_element(int eb, int t, int nx) {
  if (nx != 32) return eb * kWbThreads + t;
  const int w = t >> 5, q = (t >> 3) & 3, e = t & 7;
  const int mx = 8 * (w & 3) + 2 * q + (e & 1), my = 4 * (w >> 2) + (e >> 1);
  return (eb * 8 + my) * 32 + mx;
}

template <int WT>
__global__ void __launch_bounds__(kWbThreads, 2) k_synth_wb(SynthWbArgs a) {
  extern __shared__ __align__(16) uint8_t wb_smem[];
  const int nx = a.nx, ny = a.ny, M = nx * ny, U = a.n_phases, UF = a.uf;
  float4* s_tab = reinterpret_cast<float4*>(wb_smem);
  float2* s_ey = reinterpret_cast<float2*>(s_tab + a.n_tab);  // [kSub][nx]: c_k exp(j 2 pi pol uy (mx - cx))
  float2* s_ez = s_ey + kSub * nx;                            // [kSub][ny]
  float* s_dy = reinterpret_cast<float*>(s_ez + kSub * ny);   // [kSub][nx]: delay of column mx in entries
  float* s_dz = s_dy + kSub * nx;                             // [kSub][ny]
  float* s_x = s_dz + kSub * ny;                              // [kSub]: entry of the window's first row
  int* s_n = reinterpret_cast<int*>(s_x + kSub);              // [kSub]: the window's first row
  for (int i = threadIdx.x; i < a.n_tab; i += blockDim.x) s_tab[i] = __ldg(&a.tab[i]);
  pdl_wait();

  const int64_t H = *a.n_valid;
  const int n_eb = (M + kWbThreads - 1) / kWbThreads;
  const int64_t target = (int64_t)gridDim.x * 4;
  int64_t chunk = ((H * n_eb * U + target - 1) / target + kSub - 1) / kSub * kSub;
  if (chunk < kSub) chunk = kSub;
  if (chunk > 8192) chunk = 8192;
  const int64_t n_chunks = (H + chunk - 1) / chunk;
  const int64_t n_items = n_chunks * n_eb * U;
  const int tid = threadIdx.x;
  const float cx = 0.5f * (float)(nx - 1), cy = 0.5f * (float)(ny - 1);
  const int span = (WT - 1) * UF + 1;  // entries one (hit, element) reads from x0 on

  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int phase = (int)(item % U);
    const int64_t rest = item / U;
    const int eb = (int)(rest % n_eb);
    const int64_t c = rest / n_eb;
    const int m = wb_element(eb, tid, nx);
    const bool act = m < M;
    const int mx = act ? m % nx : 0, my = act ? m / nx : 0;
    const int64_t h0 = c * chunk, h1 = min(h0 + chunk, H);
    float2* S = a.S + (int64_t)phase * a.phase_stride;
    const float x_phase = a.tab_x0 + (float)(phase * a.f);
    float2 acc[WT];
#pragma unroll
    for (int i = 0; i < WT; ++i) acc[i] = make_float2(0.f, 0.f);
    bool open = false;
    int base = 0;

    // adds the window's first row into S and slides the window by one row
    auto shift = [&]() {
      if (base >= 0 && act) {
        float* dst = reinterpret_cast<float*>(S + (int64_t)base * M + m);
        asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(dst), "f"(acc[0].x), "f"(acc[0].y) : "memory");
      }
#pragma unroll
      for (int r = 0; r < WT - 1; ++r) acc[r] = acc[r + 1];
      acc[WT - 1] = make_float2(0.f, 0.f);
      ++base;
    };

    for (int64_t s0 = h0; s0 < h1; s0 += kSub) {
      const int nsub = (int)(h1 - s0 < kSub ? h1 - s0 : kSub);
      __syncthreads();
      const int per_hit = nx + ny;
      for (int idx = tid; idx < nsub * per_hit; idx += kWbThreads) {
        const int k = idx / per_hit, j = idx % per_hit;
        const HitRec& h = a.hits_sorted[s0 + k];
        if (j == 0) {
          s_n[k] = h.nglob - a.e1;
          s_x[k] = fmaf(h.u0, (float)UF, x_phase);
        }
        float sn, cs;
        if (j < nx) {
          const float q = (float)j - cx;
          sincospif(2.0f * a.pitch_over_lambda * q * h.uy, &sn, &cs);
          s_ey[k * nx + j] = make_float2(h.cr * cs - h.ci * sn, h.cr * sn + h.ci * cs);
          s_dy[k * nx + j] = a.pitch_uf * h.uy * q;
        } else {
          const int jj = j - nx;
          const float q = (float)jj - cy;
          sincospif(2.0f * a.pitch_over_lambda * q * h.uz, &sn, &cs);
          s_ez[k * ny + jj] = make_float2(cs, sn);
          s_dz[k * ny + jj] = a.pitch_uf * h.uz * q;
        }
      }
      __syncthreads();
      for (int k = 0; k < nsub; ++k) {
        const int g = s_n[k];
        if (!open) { base = g; open = true; }
        if (g - base >= WT) {
#pragma unroll
          for (int i = 0; i < WT; ++i) shift();
          base = g;
        }
        while (base < g) shift();
        if (!act) continue;
        const float2 ey = s_ey[k * nx + mx], ez = s_ez[k * ny + my];
        const float2 P = make_float2(ey.x * ez.x - ey.y * ez.y, ey.x * ez.y + ey.y * ez.x);
        const float x0 = s_x[k] + s_dy[k * nx + mx] + s_dz[k * ny + my];
        const float fl = floorf(x0);
        const float f = x0 - fl;
        const int j0 = (int)fl;
        if (j0 < 0 || j0 + span >= a.n_tab) {
          // the table is sized on the host to cover every delay; a position outside it
          // means the bound did not hold: record it and drop the pair
          atomicOr(a.err, kErrIndex);
          continue;
        }
        const float4* t = s_tab + j0;
#pragma unroll
        for (int i = 0; i < WT; ++i) {
          const float4 v = t[i * UF];
          const float rr = fmaf(f, v.z, v.x), ri = fmaf(f, v.w, v.y);
          acc[i].x = fmaf(P.x, rr, fmaf(-P.y, ri, acc[i].x));
          acc[i].y = fmaf(P.x, ri, fmaf(P.y, rr, acc[i].y));
        }
      }
    }
    if (open) {
#pragma unroll
      for (int i = 0; i < WT; ++i) shift();
    }
  }
}

// Pulse autocorrelation table R(u), u in [-T_p, T_p], kRTab intervals, evaluated in
// FP64 from the closed form: the Hann window as three complex exponentials turns
// R(u) into nine exponential integrals over the overlap of the two pulse supports.
__device__ inline double sinc_d(double x) { return fabs(x) < 1e-4 ? 1.0 - x * x / 6.0 : sin(x) / x; }
__device__ double2 pulse_acf(double u, double T, double B) {
  if (!(fabs(u) < T)) return make_double2(0.0, 0.0);
  const double kappa = B / T, Om = 2.0 * kPi / T, E = 3.0 * T / 8.0;
  const double L = fmax(-T / 2, -T / 2 - u), U = fmin(T / 2, T / 2 - u);
  double sr = 0.0, si = 0.0;
  for (int aa = -1; aa <= 1; ++aa) {
    for (int bb = -1; bb <= 1; ++bb) {
      double ca = aa == 0 ? 0.5 : 0.25, cb = bb == 0 ? 0.5 : 0.25;
      double beta = (aa + bb) * Om + 2.0 * kPi * kappa * u;
      double mag = (U - L) * sinc_d(beta * (U - L) / 2);
      double ph = beta * (U + L) / 2 + aa * Om * u;
      sr += ca * cb * mag * cos(ph);
      si += ca * cb * mag * sin(ph);
    }
  }
  double ph0 = kPi * kappa * u * u;
  double c0 = cos(ph0), s0 = sin(ph0);
  return make_double2((c0 * sr - s0 * si) / E, (c0 * si + s0 * sr) / E);
}
__global__ void k_rtab(float2* tab, int n_int, int guard, double T, double B) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n_int + 2 * guard) return;
  const double2 r = pulse_acf(-T + 2.0 * T * (double)(i - guard) / (double)n_int, T, B);
  tab[i] = make_float2((float)r.x, (float)r.y);
}

// Fine-grid table of the wideband synthesis: entry i holds R at v_i = v_lo + i du range
// samples and the step to entry i + 1 (FP64 evaluation, FP32 storage).
__global__ void k_wtab(float4* tab, int n, double v_lo, double du, double dt, double T, double B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 r0 = pulse_acf((v_lo + i * du) * dt, T, B);
  const double2 r1 = pulse_acf((v_lo + (i + 1) * du) * dt, T, B);
  const float2 f0 = make_float2((float)r0.x, (float)r0.y);
  tab[i] = make_float4(f0.x, f0.y, (float)r1.x - f0.x, (float)r1.y - f0.y);
}

// S (FP32, padded rows) -> 16-bit GEMM operand X [n_pings * nr_x][k_pad], interleaved
// (re, im) per element; FP32 form also writes the residual lo = x - hi.
__global__ void k_absmax(const float2* S, int32_t nr, int32_t nr_pad, int32_t M, float* gain) {
  int p = blockIdx.y;
  float mx = 0.f;
  int64_t n = (int64_t)nr * M;
  const float2* base = S + ((int64_t)p * nr_pad + kPad) * M;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float2 v = base[i];
    mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(gain + p), __float_as_int(mx));
}

// One CTA per range row (ping p, sample n): the row's M complex echoes become the GEMM's
// 16-bit operand row(s), four elements (two 16-byte loads, one 16-byte store per part)
// per thread step; rows whose M is not a multiple of 4 take the scalar path.
__device__ __forceinline__ uint32_t cvt_pair(float x, float y, int mode, float gn, uint32_t* lo) {
  if (mode == SONAR_FP16) {
    __half2 h = __floats2half2_rn(x * gn, y * gn);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __nv_bfloat162 hi = __floats2bfloat162_rn(x, y);
  if (mode == SONAR_FP32) {
    const float2 hf = __bfloat1622float2(hi);
    __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    *lo = *reinterpret_cast<uint32_t*>(&l);
  }
  return *reinterpret_cast<uint32_t*>(&hi);
}

__global__ void __launch_bounds__(256) k_convert(ConvertArgs a) {
  pdl_wait();
  // row r of the grid: phase s, ping p, operand row j = sample j - x_guard
  const int rows = a.nr + 2 * a.x_guard;
  const int r = blockIdx.x;
  const int sp = r / rows, j = r - sp * rows;
  const int s = sp / a.n_pings, p = sp - s * a.n_pings;
  const int n = j - a.x_guard;
  const int M = a.M;
  const float2* src = a.S + s * a.phase_stride + ((int64_t)p * a.nr_pad + kPad + n) * M;
  const int64_t dst0 = ((int64_t)sp * a.x_rows + j) * a.k_pad;  // 16-bit units
  uint16_t* xh = reinterpret_cast<uint16_t*>(a.x_hi) + dst0;
  uint16_t* xl = reinterpret_cast<uint16_t*>(a.x_lo) + dst0;
  const float gn = a.mode == SONAR_FP16 ? a.gain[p] : 1.0f;
  if ((M & 3) == 0) {
    for (int m = threadIdx.x * 4; m < M; m += blockDim.x * 4) {
      const float4 v0 = __ldg(reinterpret_cast<const float4*>(src + m));
      const float4 v1 = __ldg(reinterpret_cast<const float4*>(src + m + 2));
      uint4 h, l = make_uint4(0u, 0u, 0u, 0u);
      h.x = cvt_pair(v0.x, v0.y, a.mode, gn, &l.x);
      h.y = cvt_pair(v0.z, v0.w, a.mode, gn, &l.y);
      h.z = cvt_pair(v1.x, v1.y, a.mode, gn, &l.z);
      h.w = cvt_pair(v1.z, v1.w, a.mode, gn, &l.w);
      *reinterpret_cast<uint4*>(xh + 2 * m) = h;
      if (a.mode == SONAR_FP32) *reinterpret_cast<uint4*>(xl + 2 * m) = l;
    }
  } else {
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
      const float2 v = src[m];
      uint32_t l = 0u;
      const uint32_t h = cvt_pair(v.x, v.y, a.mode, gn, &l);
      *reinterpret_cast<uint32_t*>(xh + 2 * m) = h;
      if (a.mode == SONAR_FP32) *reinterpret_cast<uint32_t*>(xl + 2 * m) = l;
    }
  }
}

// Power-of-two gain so that the largest |component| lands near 2^14 in FP16.
__global__ void k_gain_pow2(float* gain, int n, int mode) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (mode != SONAR_FP16) { gain[p] = 1.0f; return; }
  float mx = gain[p];
  int e = 0;
  if (mx > 0.f) frexpf(mx, &e);
  gain[p] = ldexpf(1.0f, 14 - e);
}


// ----------------------------------------------------------------- raw series, matched filter
// The transmitted pulse p(t) = w(t) exp(j pi (B/T) t^2) on |t| <= T/2, Hann w = (1 + cos(2 pi
// t / T)) / 2 (Sec. II.B), evaluated in FP64 once per parameter set.
__device__ double2 pulse_p(double t, double T, double B) {
  if (!(fabs(t) <= T / 2)) return make_double2(0.0, 0.0);
  const double w = 0.5 * (1.0 + cos(2.0 * kPi * t / T)), ph = kPi * (B / T) * t * t;
  return make_double2(w * cos(ph), w * sin(ph));
}

// Pulse tables of phase blockIdx.y on the grid of the autocorrelation tables (entry i at
// u = -T + 2 T (i - guard) / n_int), shifted by s dt / U.
__global__ void k_ptab(float2* tab, int n_int, int guard, double T, double B, double dt, int U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, s = blockIdx.y;
  if (i > n_int + 2 * guard) return;
  const double u = -T + 2.0 * T * (double)(i - guard) / (double)n_int;
  const double2 v = pulse_p(u + s * dt / U, T, B);
  tab[(int64_t)s * (n_int + 2 * guard + 1) + i] = make_float2((float)v.x, (float)v.y);
}

__global__ void k_mftaps(float2* taps, int U, int D, double T, double B, double dt) {
  const int d = (int)threadIdx.x - D, s = blockIdx.x;
  if (d > D) return;
  const double2 v = pulse_p(d * dt + s * dt / U, T, B);
  const double g = dt / (U * (3.0 * T / 8.0));
  taps[s * (2 * D + 1) + D + d] = make_float2((float)(g * v.x), (float)(-g * v.y));
}

// y_m(t_n) = sum over the U phases s and the offsets |d| <= D of r_m(t_{n+d} + s dt / U)
// taps[s][D + d]: the rectangle rule of (1/E) int r(t) conj(p(t - t_n)) dt on the raw
// samples. A thread owns one element and kMfRows consecutive samples of a ping; the raw
// rows it reads repeat across its samples and stay in L1.
constexpr int kMfRows = 16;
__global__ void __launch_bounds__(128) k_mfilter(MfArgs a) {
  pdl_wait();
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.M) return;
  const int nblk = (a.nr + kMfRows - 1) / kMfRows;
  const int p = blockIdx.y / nblk, n0 = (blockIdx.y % nblk) * kMfRows;
  const int64_t base = ((int64_t)p * a.nr_pad + kPad) * a.M + m;
  const int n1 = min(n0 + kMfRows, a.nr);
  for (int n = n0; n < n1; ++n) {
    float yr = 0.f, yi = 0.f;
    for (int s = 0; s < a.U; ++s) {
      const float2* src = a.raw + s * a.phase_stride + base + (int64_t)n * a.M;
      const float2* h = a.taps + s * (2 * a.D + 1) + a.D;
      for (int d = -a.D; d <= a.D; ++d) {
        const float2 r = __ldg(src + (int64_t)d * a.M), t = __ldg(h + d);
        yr = fmaf(r.x, t.x, fmaf(-r.y, t.y, yr));
        yi = fmaf(r.x, t.y, fmaf(r.y, t.x, yi));
      }
    }
    a.S[base + (int64_t)n * a.M] = make_float2(yr, yi);
  }
}

}  // namespace

cudaError_t launch_bin(const HitRec* hits, const unsigned long long* n_hits, int32_t n_bins, int32_t* counts,
                       int32_t* offsets, const int32_t* rank, HitRec* sorted, int32_t* sorted_n, int sm_count,
                       int32_t* bounds, int bounds_g, int row_cost, cudaStream_t st) {
  cudaError_t e = launch_pdl(k_scan, dim3(1), dim3(1024), 0, st, (const int32_t*)counts, n_bins, offsets, counts,
                             bounds, bounds_g, row_cost);
  if (e != cudaSuccess) return e;
  e = launch_pdl(k_scatter, dim3(sm_count * 8), dim3(256), 0, st, hits, n_hits, n_bins, (const int32_t*)offsets, rank,
                 sorted, sorted_n);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_synth(const SynthArgs& a, int sm_count, cudaStream_t st) {
  const int32_t* total = a.n_valid;  // offsets[n_bins] of the binning step
  cudaError_t e;
  if (a.taps <= 8) e = launch_pdl(k_synth<8>, dim3(sm_count), dim3(kThreads), 0, st, a, total);
  else if (a.taps <= 12) e = launch_pdl(k_synth<12>, dim3(sm_count), dim3(kThreads), 0, st, a, total);
  else e = launch_pdl(k_synth<16>, dim3(sm_count), dim3(kThreads), 0, st, a, total);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_ptab(float2* ptab, float2* ptab_s, float2* taps, int32_t U, int32_t D, double pulse, double bw,
                        double dt, cudaStream_t st) {
  k_ptab<<<dim3((kRTab + 1 + 255) / 256, U), 256, 0, st>>>(ptab, kRTab, 0, pulse, bw, dt, U);
  k_ptab<<<dim3((kRTabS + 5 + 255) / 256, U), 256, 0, st>>>(ptab_s, kRTabS, 2, pulse, bw, dt, U);
  k_mftaps<<<U, 2 * D + 1, 0, st>>>(taps, U, D, pulse, bw, dt);
  return cudaGetLastError();
}

cudaError_t launch_mfilter(const MfArgs& a, cudaStream_t st) {
  const int nblk = (a.nr + kMfRows - 1) / kMfRows;
  return launch_pdl(k_mfilter, dim3((unsigned)ceil_div(a.M, 128), (unsigned)(a.n_pings * nblk)), dim3(128), 0, st,
                    a);
}

size_t synth_wb_smem(const SynthWbArgs& a) {
  return (size_t)a.n_tab * sizeof(float4) + (size_t)kSub * (a.nx + a.ny) * (sizeof(float2) + sizeof(float)) +
         (size_t)kSub * (sizeof(float) + sizeof(int));
}
constexpr int kWbSmemMax = 160 * 1024;

cudaError_t prepare_synth_wb() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_synth_wb<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWbSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(k_synth_wb<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWbSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(k_synth_wb<20>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWbSmemMax))) return e;
  return cudaFuncSetAttribute(k_synth_wb<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWbSmemMax);
}

cudaError_t launch_synth_wb(const SynthWbArgs& a, int wt, int sm_count, cudaStream_t st) {
  if (a.nx > 64 || a.ny > 64 || a.n_phases < 1) return cudaErrorInvalidValue;
  const size_t smem = synth_wb_smem(a);
  if (smem > (size_t)kWbSmemMax) return cudaErrorInvalidValue;
  const dim3 grid(2 * sm_count), block(kWbThreads);
  switch (wt) {
    case 12: return launch_pdl(k_synth_wb<12>, grid, block, smem, st, a);
    case 16: return launch_pdl(k_synth_wb<16>, grid, block, smem, st, a);
    case 20: return launch_pdl(k_synth_wb<20>, grid, block, smem, st, a);
    case 24: return launch_pdl(k_synth_wb<24>, grid, block, smem, st, a);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_wtab(float4* tab, int32_t n, double v_lo, double du, double dt, double pulse, double bw,
                        cudaStream_t st) {
  k_wtab<<<(n + 255) / 256, 256, 0, st>>>(tab, n, v_lo, du, dt, pulse, bw);
  return cudaGetLastError();
}

cudaError_t launch_rtab(float2* rtab, float2* rtab_s, double pulse, double bw, cudaStream_t st) {
  k_rtab<<<(kRTab + 1 + 255) / 256, 256, 0, st>>>(rtab, kRTab, 0, pulse, bw);
  k_rtab<<<(kRTabS + 5 + 255) / 256, 256, 0, st>>>(rtab_s, kRTabS, 2, pulse, bw);
  return cudaGetLastError();
}

cudaError_t launch_convert(const ConvertArgs& a, int sm_count, cudaStream_t st) {
  if (a.mode == SONAR_FP16) {
    cudaError_t e = cudaMemsetAsync(a.gain, 0, sizeof(float) * a.n_pings, st);
    if (e != cudaSuccess) return e;
    k_absmax<<<dim3(sm_count, a.n_pings), 256, 0, st>>>(a.S, a.nr, a.nr_pad, a.M, a.gain);
  }
  if (a.mode == SONAR_FP16) k_gain_pow2<<<(a.n_pings + 63) / 64, 64, 0, st>>>(a.gain, a.n_pings, a.mode);
  if (a.x_guard > kPad || a.nr + 2 * a.x_guard > a.x_rows) return cudaErrorInvalidValue;
  cudaError_t ce = launch_pdl(k_convert, dim3(a.n_phases * a.n_pings * (a.nr + 2 * a.x_guard)), dim3(256), 0, st, a);
  if (ce != cudaSuccess) return ce;
  return cudaGetLastError();
}

}  // namespace sonar
