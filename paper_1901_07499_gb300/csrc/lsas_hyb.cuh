// lsas_hyb.cuh -- fused receiver for N = 1024 (sc16 input) with the second
// FFT pass on the tensor cores.
//
// With n = 32 n1 + n2 and k = k1 + 32 k2, the N = 1024 point DFT of one
// antenna-symbol row (Sec. II-C: one FFT per antenna and OFDM symbol) is
//   pass 1   T[k1][n2] = W_1024^(n2 k1) sum_n1 x[32 n1 + n2] W_32^(n1 k1)
//   pass 2   Y[k1 + 32 k2] = sum_n2 T[k1][n2] W_32^(n2 k2)
// Pass 1 runs on the CUDA cores exactly as in the per-warp kernel: lane n2
// of a warp holds x[32 n1 + n2] for all n1 in registers, transforms them and
// applies the twiddles (scaled by 2^-5, which keeps every value in fp16 range
// and makes pass 2 produce the unitary transform directly).  The lane then
// owns column n2 of T.  Pass 2 is a complex GEMM on tcgen05: the four warps
// of a quad (one per TMEM lane quarter) store their rows' T as the A operand
// of one M = 128 MMA (rows = the four FFTs' k1, K = n2 re | n2 im), in the
// MN-major layout, so that a lane's column lands as one 16-byte chunk per 8
// rows: the transpose between the passes costs no shared-memory exchange.
// Each value is split into fp16 hi = fp16(v) and lo = fp16(v - hi), and the
// product with the fp16 hi+lo DFT-32 operand is summed as
// A_hi B_hi + A_lo B_hi + A_hi B_lo (fp32 accumulation in TMEM; the dropped
// lo*lo term is ~2^-22 relative).  The accumulator row of lane k1 then holds
// Y[k1 + 32 k2] for all k2 -- the same subcarriers the per-warp kernel's
// lane owns -- and LS (Sec. II-C), the MRC sums (Sec. II-C, III) and the
// demapper follow as there.
//
// Pipeline per warp and step (one antenna-symbol row): stage (bulk copy,
// the CP removal of Sec. II-B as addressing) -> pass 1 -> store the A rows
// of this step (two A buffers per quad) -> wait for the quad's previous MMA
// and run LS or MRC of that step straight from its accumulator rows ->
// arrive on the quad's "operands ready" barrier (the last warp to arrive
// issues the 12 MMAs of the step).  So a step's MMA runs while its warps
// stage and transform the next one.  Every wait is bounded.
#pragma once

#include <cuda_fp16.h>

#include "lsas_kernels.cuh"
#include "lsas_warp.cuh"

namespace lsas {

constexpr int kHyWarps = 8;                 // two quads of four warps
constexpr int kHyThreads = 32 * kHyWarps;
constexpr int kHySlots = 2;                 // staging ring depth per warp
constexpr int kHyRow = 1024 * 4;            // one sc16 row of N = 1024
constexpr int kHyImg = 128 * 64 * 2;        // one fp16 A image: 128 rows x K = 64
constexpr int kHyDgMax = 2;                 // data symbols per group (TMEM)
// tensor memory columns (all 512 of the SM are allocated)
constexpr int kHyAcc = 0;                   // quad Q accumulator at Q * 64
constexpr int kHyWarpCol = 128;             // warp w: E, then P per data symbol,
constexpr int kHyWarpCols = 160;            //   at 128 + (w >> 2) * 160 in its lane quarter
// shared memory
constexpr int kHyBarStage = 0;              // [warp][slot] staging mbarriers
constexpr int kHyBarReady = kHyWarps * kHySlots * 8;   // [quad] operands ready
constexpr int kHyBarDone = kHyBarReady + 16;           // [quad] MMA done
constexpr int kHyTmemAddr = kHyBarDone + 16;
constexpr int kHyAbort = kHyTmemAddr + 4;
constexpr int kHyTag = kHyAbort + 4;        // [quad] next step whose MMAs are unclaimed
constexpr int kHyB = 1024;                  // DFT-32 operand images hi, lo (8 KB each)
constexpr int kHyIe = kHyB + 2 * 8192;      // 1/E per subcarrier
constexpr int kHyCodes = kHyIe + 1024 * 4;  // demapped codes [dg][N]
constexpr int kHyA = kHyCodes + kHyDgMax * 1024;       // A images [quad][buf][hi, lo]
constexpr int kHyTwS = kHyA + 2 * 2 * 2 * kHyImg;      // pass twiddles [k1][n2], x 2^-5
constexpr int kHyStage = kHyTwS + 32 * 32 * 8;         // staging [warp][slot]
constexpr int kHySmem = kHyStage + kHyWarps * kHySlots * kHyRow;
static_assert(kHyA % 1024 == 0 && kHyStage % 1024 == 0 && kHyTwS % 16 == 0, "aligned regions");
static_assert(kHySmem <= 232448, "fits one SM");

#ifdef __CUDACC__

// byte offset of element (row m, k) of an MN-major A image (128 rows, K = 64):
// core matrices of 8 K x 16 bytes (8 rows), row groups 128 bytes apart, K
// groups 2048 bytes apart
__host__ __device__ constexpr int hy_aoff(int m, int k) {
  return (m >> 3) * 128 + (k >> 3) * 2048 + (k & 7) * 16 + (m & 7) * 2;
}

// fp32 -> (hi, lo) fp16 pair words for two values: hi keeps the top 11
// significant bits (exact in fp16 for normal values), lo = v - hi exactly,
// rounded to fp16
__device__ __forceinline__ void hy_split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const float ha = __uint_as_float(__float_as_uint(a) & 0xFFFFE000u);
  const float hb = __uint_as_float(__float_as_uint(b) & 0xFFFFE000u);
  const __half2 h = __floats2half2_rn(ha, hb);
  const __half2 l = __floats2half2_rn(a - ha, b - hb);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Issue one step's bulk copy (one antenna-symbol row) into a slot: lane 0
// registers the bytes (none for an antenna past M: the phase still completes).
__device__ __forceinline__ void hy_issue(const KParams& p, int f, int m, int s, bool valid,
                                         unsigned char* slot, uint32_t bar, uint64_t pol,
                                         int lane) {
  if (lane == 0) {
    mbar_expect_tx(bar, valid ? kHyRow : 0);
    if (valid) bulk_load(smem_u32(slot), row_ptr<10, false>(p, f, m, s), kHyRow, bar, pol);
  }
}

// Channel energy of one antenna added to the lane's 32 TMEM columns at tE.
__device__ __forceinline__ void hy_add_energy(uint32_t tE, const float2 (&h)[32]) {
  tmem_wait_st();
#pragma unroll
  for (int e0 = 0; e0 < 32; e0 += 16) {
    float acc[16];
    Tmem<16>::ld(tE + e0, acc);
    tmem_wait_ld();
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = fmaf(h[e0 + e].x, h[e0 + e].x, fmaf(h[e0 + e].y, h[e0 + e].y, acc[e]));
    Tmem<16>::st(tE + e0, acc);
  }
}

// Walks one warp's steps in order: data-symbol group g, antenna chunk lc,
// item it (the pilot first where the group transforms it).
struct HyCursor {
  int g, lc, it, items, nch;
  __device__ void start(const KParams& p, int g0, int nch_) {
    g = g0;
    lc = 0;
    it = 0;
    nch = nch_;
    items = hy_items(p, g);
  }
  __device__ static int hy_items(const KParams& p, int g) {
    const int nd = min(p.dg, p.D - g * p.dg);
    return nd + ((fft_pilot(p) && (g == 0 || p.group_z)) ? 1 : 0);
  }
  __device__ bool pilot_here(const KParams& p) const { return fft_pilot(p) && (g == 0 || p.group_z); }
  __device__ int symbol(const KParams& p) const {
    return witem_symbol(p, pilot_here(p), g * p.dg, it);
  }
  __device__ void next(const KParams& p) {
    if (++it < items) return;
    it = 0;
    if (++lc < nch) return;
    lc = 0;
    ++g;
    items = hy_items(p, g < p.groups ? g : 0);
  }
};

template <bool FC32>
__global__ void __launch_bounds__(kHyThreads, 1) hyb_kernel(const KParams p) {
  static_assert(!FC32, "the tensor-core kernel stages sc16 rows");
  constexpr int N = 1024;
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int Q = warp >> 2;      // quad
  const int q = warp & 3;       // TMEM lane quarter (= warp % 4)
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kHyBarStage) + warp * kHySlots;
  const uint32_t bar_ready = smem_u32(smem + kHyBarReady + 8 * Q);
  const uint32_t bar_done = smem_u32(smem + kHyBarDone + 8 * Q);
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(smem + kHyTmemAddr);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kHyAbort);
  int* tag = reinterpret_cast<int*>(smem + kHyTag) + Q;
  float* ie_s = reinterpret_cast<float*>(smem + kHyIe);
  uint8_t* codes = smem + kHyCodes;
  const float2* tws = reinterpret_cast<const float2*>(smem + kHyTwS);
  unsigned char* stage = smem + kHyStage + warp * kHySlots * kHyRow;
  unsigned char* aimg = smem + kHyA + Q * 2 * 2 * kHyImg;   // [buf][hi, lo]

  // DFT-32 operand images (hi, lo) and the pass twiddles W_1024^(n2 k1) 2^-5
  // ([k1][n2]; exact scaling) into shared memory
  {
    const uint4* s = static_cast<const uint4*>(p.tc_w1);
    uint4* d = reinterpret_cast<uint4*>(smem + kHyB);
    for (int i = tid; i < 2 * 8192 / 16; i += kHyThreads) d[i] = __ldg(s + i);
    float2* t = reinterpret_cast<float2*>(smem + kHyTwS);
    for (int i = tid; i < 32 * 32; i += kHyThreads) {
      const float2 w = __ldg(p.twP + i);   // [r][j] = W_1024^(j r)
      t[i] = make_float2(w.x * 0.03125f, w.y * 0.03125f);
    }
  }
  if (tid == 0) {
    *abort_flag = 0;
    reinterpret_cast<int*>(smem + kHyTag)[0] = 0;
    reinterpret_cast<int*>(smem + kHyTag)[1] = 0;
    for (int i = 0; i < kHyWarps * kHySlots; ++i)
      mbar_init(smem_u32(smem + kHyBarStage + 8 * i), 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(smem + kHyBarReady + 8 * i), 4);
      mbar_init(smem_u32(smem + kHyBarDone + 8 * i), 1);
    }
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_base), 512);
  fence_proxy_async();
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t tbase = *tmem_base;
  const uint32_t tlane = static_cast<uint32_t>(32 * q) << 16;
  const uint32_t tacc = tbase + tlane + kHyAcc + 64 * Q;        // this warp's accumulator rows
  const uint32_t tE = tbase + tlane + kHyWarpCol + Q * kHyWarpCols;
  const uint32_t tP = tE + 32;                                  // data symbol dl at tP + 64 dl

  uint64_t pol = 0;
  if (lane == 0) pol = evict_first_policy();
  pol = __shfl_sync(0xffffffffu, pol, 0);

  // chunks (antennas) of this warp: warp + 8 lc; every warp of a quad runs as
  // many steps as the quad's first warp (past M the rows are zero)
  const int nchQ = 4 * Q < p.chunks ? (p.chunks - 1 - 4 * Q) / kHyWarps + 1 : 0;
  const int g_lo = p.group_z ? static_cast<int>(blockIdx.z) : 0;
  const int g_hi = p.group_z ? g_lo + 1 : p.groups;
  // staging: issue cursor and the number of steps still to issue
  HyCursor ic;
  ic.start(p, g_lo, nchQ);
  int to_issue = 0;
  for (int g = g_lo; g < g_hi; ++g) to_issue += nchQ * HyCursor::hy_items(p, g);
  int issued = 0;
  int slot = 0, phase = 0;   // ring slot and mbarrier phase of the next step to consume
  int step = 0;              // this warp's (= its quad's) step counter
  if (nchQ > 0) {
    fence_proxy_async();
    for (int s = 0; s < kHySlots && to_issue > 0; ++s, --to_issue) {
      const int m = warp + ic.lc * kHyWarps;
      hy_issue(p, f, m, ic.symbol(p), m < p.M, stage + s * kHyRow,
               smem_u32(&bars[s]), pol, lane);
      // test hook: the first staging phase of block 0 also waits for 16
      // bytes that no copy delivers, so its bounded wait runs out
      if (p.fault == 1 && blockIdx.x == 0 && warp == 0 && s == 0 && lane == 0)
        mbar_expect_tx_only(smem_u32(&bars[0]), 16);
      ++issued;
      ic.next(p);
    }
  }

  float zero[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) zero[i] = 0.f;
  float2 h[32];   // channel of the antenna whose step is being combined
#pragma unroll
  for (int e = 0; e < 32; ++e) h[e] = make_float2(0.f, 0.f);

  for (int g = g_lo; g < g_hi; ++g) {
    const int nd = min(p.dg, p.D - g * p.dg);
    const int d0 = g * p.dg;
    const bool pilot_here = fft_pilot(p) && (g == 0 || p.group_z);
    const int items = nd + (pilot_here ? 1 : 0);
    const bool first_e = (g == g_lo);   // this block accumulates the channel energy
    if (first_e) {
      Tmem<16>::st(tE, zero);
      Tmem<16>::st(tE + 16, zero);
    }
    for (int c = 0; c < 64 * nd; c += 16) Tmem<16>::st(tP + c, zero);
    const int gsteps = nchQ * items;
    // the step being combined (the previous one): its item and antenna
    int pit = -1, pm = 0;
    int lc = 0, it = 0;   // chunk and item of the step being transformed
    for (int gs = 0; gs <= gsteps; ++gs) {
      const bool have = gs < gsteps;     // a step to transform (else: drain)
      const int m = warp + lc * kHyWarps;
      const bool valid = m < p.M;
      if (have) {
        // ---- stage
        float2 v[32];
        wait_slot(smem_u32(&bars[slot]), phase, abort_flag, p.status);
        if (valid) {
          load_row<10, false>(v, stage + slot * kHyRow, lane, false);
        } else {
#pragma unroll
          for (int r = 0; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
        }
        __syncwarp();
        if (to_issue > 0 && !*abort_flag) {
          fence_proxy_async();
          const int mi = warp + ic.lc * kHyWarps;
          hy_issue(p, f, mi, ic.symbol(p), mi < p.M, stage + slot * kHyRow,
                   smem_u32(&bars[slot]), pol, lane);
          --to_issue;
          ++issued;
          ic.next(p);
        }
        if (++slot == kHySlots) {
          slot = 0;
          phase ^= 1;
        }
        // ---- pass 1 (radix 32 over n1) and the pass twiddles
        dft<32>(v, p);
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const float2 w = tws[r * 32 + lane];
          const float2 a = v[r];
          v[r] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
        }
        // ---- A rows of this step: row 32 q + k1, K = lane (re), 32 + lane
        // (im); buffer step & 1 was last read by the MMA of step - 2, which
        // this warp saw complete one step ago
        unsigned char* ahi = aimg + (step & 1) * 2 * kHyImg;
        unsigned char* alo = ahi + kHyImg;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          uint32_t hr[4], lr[4], hi_[4], li[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            hy_split2(v[8 * i + 2 * j].x, v[8 * i + 2 * j + 1].x, hr[j], lr[j]);
            hy_split2(v[8 * i + 2 * j].y, v[8 * i + 2 * j + 1].y, hi_[j], li[j]);
          }
          const int ore = hy_aoff(32 * q + 8 * i, lane);
          const int oim = hy_aoff(32 * q + 8 * i, 32 + lane);
          *reinterpret_cast<uint4*>(ahi + ore) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
          *reinterpret_cast<uint4*>(alo + ore) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
          *reinterpret_cast<uint4*>(ahi + oim) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
          *reinterpret_cast<uint4*>(alo + oim) = make_uint4(li[0], li[1], li[2], li[3]);
        }
      }
      // ---- LS or MRC of the previous step, straight from its accumulator
      // rows (before this step's MMAs may overwrite them)
      if (gs > 0) {
        // (waited even after an abort: no MMA may still run when the block
        // releases its tensor memory)
        if (!mbar_wait_bounded(bar_done, (step - 1) & 1)) {
          *abort_flag = 1;
          latch(p.status, kStTimeout);
        }
        tmem_fence_after();
        const bool valid_prev = pm < p.M;
        if (pilot_here && pit == 0) {
          // LS estimate H = Y conj(X) / |X|^2 (xinv carries 1/sqrt(N); Y here
          // is the unitary transform)
          const size_t hrow =
              (static_cast<size_t>(f) * p.Mtot + p.m0 + blockIdx.y * p.shard_y + pm) * N;
          const bool write_h = valid_prev && (!p.group_z || blockIdx.z == 0);
#pragma unroll
          for (int e0 = 0; e0 < 32; e0 += 16) {
            float yr[16], yi[16];
            Tmem<16>::ld(tacc + e0, yr);
            Tmem<16>::ld(tacc + 32 + e0, yi);
            float2 xi[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) xi[e] = __ldg(p.xinv + lane + 32 * (e0 + e));
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float a = yr[e], b = yi[e];
              const float2 hv = make_float2((a * xi[e].x - b * xi[e].y) * 32.f,
                                            (a * xi[e].y + b * xi[e].x) * 32.f);
              h[e0 + e] = valid_prev ? hv : make_float2(0.f, 0.f);
              if (write_h) p.H_out[hrow + lane + 32 * (e0 + e)] = hv;
            }
          }
          if (first_e) hy_add_energy(tE, h);
        } else {
          const int dl = pit - (pilot_here ? 1 : 0);
          const uint32_t tp = tP + 64 * dl;
          tmem_wait_st();
#pragma unroll
          for (int e0 = 0; e0 < 32; e0 += 16) {
            float yr[16], yi[16], pr[16], pi[16];
            Tmem<16>::ld(tacc + e0, yr);
            Tmem<16>::ld(tacc + 32 + e0, yi);
            Tmem<16>::ld(tp + e0, pr);
            Tmem<16>::ld(tp + 32 + e0, pi);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float2 hh = h[e0 + e];
              pr[e] = fmaf(hh.x, yr[e], fmaf(hh.y, yi[e], pr[e]));
              pi[e] = fmaf(hh.x, yi[e], fmaf(-hh.y, yr[e], pi[e]));
            }
            Tmem<16>::st(tp + e0, pr);
            Tmem<16>::st(tp + 32 + e0, pi);
          }
        }
      }
      if (have) {
        // ---- operands of this step ready (and the accumulator read): the
        // quad's last warp to arrive issues the step's MMAs
        fence_proxy_async();
        tmem_fence_before();
        __syncwarp();
        if (lane == 0) {
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar_ready) : "memory");
          if (mbar_test_wait(bar_ready, step & 1) && atomicCAS(tag, step, step + 1) == step) {
            tmem_fence_after();
            const uint32_t a0 = smem_u32(aimg + (step & 1) * 2 * kHyImg);
            const uint32_t b0 = smem_u32(smem + kHyB);
            const uint32_t idesc = umma_idesc(64, false) | (1u << 15);   // A MN-major
            const uint32_t dacc = tbase + kHyAcc + 64 * Q;
#pragma unroll
            for (int term = 0; term < 3; ++term) {
              const uint32_t ab = a0 + (term == 1 ? kHyImg : 0);      // A lo for term 1
              const uint32_t bb = b0 + (term == 2 ? 8192 : 0);        // B lo for term 2
#pragma unroll
              for (int kc = 0; kc < 4; ++kc)
                umma_f16(dacc, umma_desc(ab + kc * 4096, 2048, 128), umma_desc(bb + kc * 256, 128, 1024),
                         idesc, (term > 0 || kc > 0) ? 1u : 0u);
            }
            umma_commit(bar_done);
          }
        }
        __syncwarp();
        // channel of this step's antenna, when it comes from memory (first
        // item of an antenna in a group without the pilot): loaded now, used
        // when this step is combined, one step later
        if (!pilot_here && it == 0) {
          const float2* Hs = fft_pilot(p) ? p.H_out : p.H_in;
          const size_t hrow = (static_cast<size_t>(f) * p.Mtot + p.m0 + blockIdx.y * p.shard_y + m) * N;
#pragma unroll
          for (int e = 0; e < 32; ++e) h[e] = valid ? Hs[hrow + lane + 32 * e] : make_float2(0.f, 0.f);
          if (first_e) hy_add_energy(tE, h);
        }
        pit = it;
        pm = m;
        ++step;
        if (++it == items) {
          it = 0;
          ++lc;
        }
      }
    }
    tmem_wait_st();
    // ---- group end: every step of the group has been combined; the A
    // images are free and hold the cross-warp reduction
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    unsigned char* red = smem + kHyA;
    if (first_e) {
      float* RE = reinterpret_cast<float*>(red);   // [NW][N]
      float e[32];
      Tmem<32>::ld(tE, e);
      tmem_wait_ld();
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) RE[warp * N + lane + 32 * cc] = e[cc];
      __syncthreads();
      for (int k = tid; k < N; k += kHyThreads) {
        float E = 0.f;
#pragma unroll
        for (int w = 0; w < kHyWarps; ++w) E += RE[w * N + k];
        if (p.mode == kModePartial) {
          if (!p.group_z || blockIdx.z == 0)
            p.E_out[(static_cast<size_t>(blockIdx.y) * gridDim.x + f) * N + k] = E;
        } else {
          const bool ok = (E > 0.f) && (E <= 3.4028234663852886e38f);
          if (!ok) latch(p.status, kStDevice);
          ie_s[k] = ok ? 1.0f / E : 0.f;
        }
      }
      __syncthreads();
    }
    float2* RP = reinterpret_cast<float2*>(red);   // [NW][2][N]
    for (int j = 0; j < nd; ++j) {
#pragma unroll
      for (int e0 = 0; e0 < 32; e0 += 16) {
        float pr[16], pi[16];
        Tmem<16>::ld(tP + 64 * j + e0, pr);
        Tmem<16>::ld(tP + 64 * j + 32 + e0, pi);
        tmem_wait_ld();
        float2* dst = RP + static_cast<size_t>(warp * kHyDgMax + j) * N;
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) dst[lane + 32 * (e0 + cc)] = make_float2(pr[cc], pi[cc]);
      }
    }
    __syncthreads();
    for (int idx = tid; idx < nd * N; idx += kHyThreads) {
      const int j = idx >> 10;
      const int k = idx & (N - 1);
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int w = 0; w < kHyWarps; ++w) s = cadd(s, RP[static_cast<size_t>(w * kHyDgMax + j) * N + k]);
      if (p.mode == kModePartial) {
        p.P_out[((static_cast<size_t>(blockIdx.y) * gridDim.x + f) * p.D + d0 + j) * N + k] = s;
      } else {
        const float ie = ie_s[k];
        const float2 z = (ie != 0.f) ? make_float2(s.x * ie, s.y * ie) : make_float2(0.f, 0.f);
        if (p.eq) p.eq[(static_cast<size_t>(f) * p.D + d0 + j) * N + k] = z;
        uint32_t code = gray(axis_level(z.x, p));
        if (p.axes == 2) code = (code << p.wbits) | gray(axis_level(z.y, p));
        codes[j * N + k] = static_cast<uint8_t>(code);
      }
    }
    __syncthreads();
    if (p.mode != kModePartial) {
      // pack: 8 consecutive subcarriers -> q bytes
      const int items8 = nd * (N / 8);
      const size_t frame_bytes = static_cast<size_t>(p.D) * N * p.q / 8;
      for (int it8 = tid; it8 < items8; it8 += kHyThreads) {
        const int dl = it8 / (N / 8);
        const int k0 = (it8 % (N / 8)) * 8;
        uint64_t acc = 0;
#pragma unroll
        for (int bb = 0; bb < 8; ++bb) acc = (acc << p.q) | codes[dl * N + k0 + bb];
        uint8_t* dst = p.bits + f * frame_bytes + (static_cast<size_t>(d0 + dl) * N + k0) * p.q / 8;
        for (int jb = 0; jb < p.q; ++jb) dst[jb] = static_cast<uint8_t>(acc >> (8 * (p.q - 1 - jb)));
      }
    }
    // the reduction area (A images) and the codes are reused by the next group
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
  }
  if (lane == 0 && *abort_flag) {
    // a wait gave up: give any copy of this warp still in flight a bounded
    // chance to land before the block's shared memory is released
    for (int s = 0; s < kHySlots && s < issued; ++s) {
      const int last = issued - 1 - ((issued - 1 - s) % kHySlots);
      (void)mbar_wait_bounded(smem_u32(&bars[last % kHySlots]), (last / kHySlots) & 1);
    }
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

#endif  // __CUDACC__

}  // namespace lsas
