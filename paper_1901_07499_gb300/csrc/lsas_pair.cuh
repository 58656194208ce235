// lsas_pair.cuh -- fused receiver kernel for N = 2048 from sc16 rows: pairs
// of warps as independent pipelines.
//
// One block per frame, four pairs of warps.  A pair is the FFT team of one
// antenna-symbol row (64 threads, 32 points each; Stockham radix 32 x 8 x 8,
// the batched FFT of Sec. II-C) and walks its own antennas m = q, q + 4, ...
// with its own staging ring (bulk copies of the CP-stripped rows: the CP
// removal of Sec. II-B done as addressing) and its own two exchange buffers.
// A step needs two barriers of the pair's 64 threads and nothing from the
// other pairs:
//   * wait for the staging slot, convert the row, radix-32 pass;
//   * middle exchange; the barrier between its write and read also tells the
//     pair that the staging slot is free, and it is refilled K steps ahead;
//     pass twiddles and four radix-8 DFTs;
//   * final exchange (second barrier), last-pass twiddles, four radix-8 DFTs;
//   * pilot: LS estimate H = Y conj(X) / |X|^2 (Sec. II-C), written out and
//     kept in registers, |H|^2 added to the channel energy; data symbol:
//     conj(H) Y (Sec. II-C) accumulated per subcarrier in the warp's own
//     tensor-memory columns.
// With two exchange buffers two barriers per step suffice: a thread writes
// the middle buffer of step s + 1 only after the final barrier of step s,
// which every thread passes after its last middle read of step s, and the
// final buffer of step s + 1 only after the middle barrier of step s + 1,
// which every thread passes after its last final read of step s.
// At a data-symbol group's end the block adds the pairs' partial sums in pair
// order through shared memory, forms z = P / E and demaps (Sec. II-B), or
// writes the block's partial sums (antenna split).
#pragma once

#include "lsas_kernels.cuh"
#include "lsas_warp.cuh"   // witem_symbol

namespace lsas {

constexpr int kPPairs = 4;                 // warp pairs per block
constexpr int kPN = 2048;                  // the one FFT length of this kernel
constexpr int kPXS = kPN + kPN / 32;       // exchange buffer (float2), one pad per 32
constexpr int kPThreads = 64 * kPPairs;
constexpr int kPOwn = 32;                  // subcarriers per thread
constexpr int kPTmemWarp = 256;            // TMEM columns per warp

// Shared memory of the pair kernel: the warp kernel's header (mbarriers
// [pair][kMaxSlots], TMEM address, abort flag), 1/E per subcarrier, the
// demapped codes of one group, the last-pass twiddles W_2048^(j r) for
// r = 1..7, j < 256, then one region per pair (staging ring of nslots rows,
// middle and final exchange).  At group ends the regions together hold the
// pairs' partial sums.
constexpr int kPTwl = 7 * 256;             // last-pass twiddles (float2)
struct PLayout {
  int ie_off, codes_off, tw_off, pair_off;
  int stage_bytes;   // one pair's ring
  int pair_bytes;    // one pair's region
  int total;
};
__host__ __device__ inline PLayout make_playout(int nslots, int dg) {
  PLayout l;
  l.ie_off = kWHeader;
  l.codes_off = l.ie_off + kPN * 4;
  l.tw_off = align_up(l.codes_off + dg * kPN, 16);
  l.pair_off = align_up(l.tw_off + kPTwl * 8, 128);
  l.stage_bytes = nslots * kPN * 4;
  l.pair_bytes = align_up(l.stage_bytes + 2 * kPXS * 8, 128);
  l.total = l.pair_off + kPPairs * l.pair_bytes;
  return l;
}
// data symbols per group that a warp's TMEM columns hold (energy + 2 per symbol)
__host__ __device__ constexpr int pgeo_dg_max() { return (kPTmemWarp - kPOwn) / (2 * kPOwn); }

#ifdef __CUDACC__

template <int LOG2N>
__global__ void __launch_bounds__(kPThreads, 1) pair_kernel(const KParams p) {
  constexpr int N = 1 << LOG2N;
  static_assert(N == kPN, "the pair kernel covers N = 2048");
  constexpr int OWN = kPOwn;
  constexpr int kRow = N * 4;   // sc16 row bytes
  using TmP = Tmem<2 * OWN>;    // one data symbol of partial sums (complex)
  using TmE = Tmem<OWN>;        // channel energy
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int q = warp >> 1;        // pair
  const int jt = tid & 63;        // FFT team thread
  const bool issuer = jt == 0;    // issues the pair's copies
  const int pbar = 1 + q;         // the pair's named barrier (0 is the block's)
  const int K = p.nslots;
  const PLayout lay = make_playout(K, p.dg);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem) + q * kMaxSlots;
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(smem + kWTmemAddr);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kWAbort);
  float* ie_s = reinterpret_cast<float*>(smem + lay.ie_off);
  uint8_t* codes = smem + lay.codes_off;
  float2* twl = reinterpret_cast<float2*>(smem + lay.tw_off);   // [r - 1][j]
  unsigned char* stage = smem + lay.pair_off + q * lay.pair_bytes;
  float2* exM = reinterpret_cast<float2*>(stage + lay.stage_bytes);   // middle exchange
  float2* exF = exM + kPXS;                                           // final exchange

  for (int i = tid; i < kPTwl; i += kPThreads) twl[i] = __ldg(p.twP + 512 + i);
  if (tid == 0) *abort_flag = 0;
  if (issuer && p.use_tma) {
    for (int s = 0; s < K; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_base), kWTmemCols);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  // this warp's columns: 256 columns of its lane quarter
  const uint32_t tE = *tmem_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                      static_cast<uint32_t>((warp >> 2) * kPTmemWarp);
  const uint32_t tP = tE + OWN;   // data symbol dl at tP + 2 OWN dl
  uint64_t pol = 0;
  if (issuer && p.use_tma) pol = evict_first_policy();
  // middle-pass twiddles of this thread, W_2048^(8 j r) for j = jt mod 32,
  // with -j W for the packed multiply (the last pass reads its own,
  // W_2048^(j r), from shared memory each step)
  float2 wm[8], wmn[8];
  wm[0] = make_float2(1.f, 0.f);
  wmn[0] = make_float2(0.f, 1.f);
#pragma unroll
  for (int r = 1; r < 8; ++r) {
    wm[r] = __ldg(p.twP + r * 32 + (jt & 31));
    wmn[r] = make_float2(-wm[r].y, wm[r].x);
  }
  float zero[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) zero[i] = 0.f;

  const int nch = q < p.chunks ? (p.chunks - 1 - q) / kPPairs + 1 : 0;
  // start the pairs of the upper half a little later, so that the two warps
  // sharing a scheduler tend to be in different phases of their steps
  if (warp >= 4) __nanosleep(1400);
  int issued = 0;  // steps whose copies this pair has issued (issuer only)
  int slot = 0;    // ring slot of the next step to consume ...
  int phase = 0;   // ... and its mbarrier phase
  // one data-symbol group per grid z index (partial mode, small batches):
  // every group's block transforms the pilot itself; group 0 alone writes H
  // and the channel energy
  const int g_lo = p.group_z ? static_cast<int>(blockIdx.z) : 0;
  const int g_hi = p.group_z ? g_lo + 1 : p.groups;
  for (int g = g_lo; g < g_hi; ++g) {
    const int nd = min(p.dg, p.D - g * p.dg);
    const int d0 = g * p.dg;
    const bool pilot_here = fft_pilot(p) && (g == 0 || p.group_z);
    const int items = nd + (pilot_here ? 1 : 0);
    if (g == g_lo) {
#pragma unroll
      for (int q0 = 0; q0 < OWN; q0 += 16) Tmem<16>::st(tE + q0, zero);
    }
    for (int dl = 0; dl < nd; ++dl) {
#pragma unroll
      for (int q0 = 0; q0 < 2 * OWN; q0 += 16) Tmem<16>::st(tP + 2 * OWN * dl + q0, zero);
    }
    // issue cursor (issuer only): local chunk and item of the next step to
    // stage, and how many steps of this group are still to be staged
    int ic = 0, iit = 0;
    int to_issue = nch * items;
    if (issuer && p.use_tma && !*abort_flag) {
      // the ring held generic data (last group's reduction): order it before
      // the copies, then fill the first K slots of this group
      fence_proxy_async();
      int is = slot;
      for (int s = 0; s < K && to_issue > 0; ++s, --to_issue) {
        const uint32_t bar = smem_u32(&bars[is]);
        mbar_expect_tx(bar, kRow);
        bulk_load(smem_u32(stage + is * kRow),
                  row_ptr<LOG2N, false>(p, f, q + ic * kPPairs, witem_symbol(p, pilot_here, d0, iit)),
                  kRow, bar, pol);
        // test hook: the first staging phase of block 0 also waits for 16
        // bytes that no copy delivers, so its bounded wait runs out
        if (p.fault == 1 && blockIdx.x == 0 && q == 0 && g == g_lo && s == 0)
          mbar_expect_tx_only(bar, 16);
        ++issued;
        is = (is + 1 == K) ? 0 : is + 1;
        if (++iit == items) {
          iit = 0;
          ++ic;
        }
      }
    }
    for (int lc = 0; lc < nch; ++lc) {
      const int m = q + lc * kPPairs;
      const size_t hrow = (static_cast<size_t>(f) * p.Mtot + p.m0 + blockIdx.y * p.shard_y + m) * N;
      float2 h[32];
      if (!pilot_here) {
        // channel from memory: given (demodulate) or written in group 0
        const float2* Hs = fft_pilot(p) ? p.H_out : p.H_in;
#pragma unroll
        for (int e = 0; e < 32; ++e) h[e] = Hs[hrow + bin_of<LOG2N>(jt, e)];
        if (g == 0) {
          float acc[OWN];
          tmem_wait_st();
          TmE::ld(tE, acc);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 32; ++e) acc[e] = fmaf(h[e].x, h[e].x, fmaf(h[e].y, h[e].y, acc[e]));
          TmE::st(tE, acc);
        }
      }
      for (int it = 0; it < items; ++it) {
        float2 v[32];
        if (p.use_tma) {
          wait_slot(smem_u32(&bars[slot]), phase, abort_flag, p.status);
          load_row<LOG2N, false>(v, stage + slot * kRow, jt, false);
        } else {
          load_row<LOG2N, false>(v, row_ptr<LOG2N, false>(p, f, m, witem_symbol(p, pilot_here, d0, it)),
                                 jt, true);
        }
        dft<32, true>(v, p);
        // middle pass: Y1[jt * 32 + r] out, Y1[j + 256 r] in (j = jt + 64 i)
#pragma unroll
        for (int r = 0; r < 32; ++r) exM[xpad(jt * 32 + r)] = v[r];
        bar_sync(pbar, 64);
        // both warps have read the staging slot: refill it K steps ahead
        if (issuer && p.use_tma && to_issue > 0 && !*abort_flag) {
          const uint32_t bar = smem_u32(&bars[slot]);
          fence_proxy_async();
          mbar_expect_tx(bar, kRow);
          bulk_load(smem_u32(stage + slot * kRow),
                    row_ptr<LOG2N, false>(p, f, q + ic * kPPairs, witem_symbol(p, pilot_here, d0, iit)),
                    kRow, bar, pol);
          ++issued;
          --to_issue;
          if (++iit == items) {
            iit = 0;
            ++ic;
          }
        }
        if (++slot == K) {
          slot = 0;
          phase ^= 1;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int j = jt + 64 * i;
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const float2 u = exM[xpad(j + 256 * r)];
            v[i * 8 + r] = (r == 0) ? u : cmulw(u, wm[r], wmn[r]);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) dft<8>(v + i * 8, p);
        final_exchange_write<LOG2N>(v, exF, jt);
        bar_sync(pbar, 64);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int j = jt + 64 * i;
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const float2 u = exF[xpad(j + 256 * r)];
            v[i * 8 + r] = (r == 0) ? u : cmul(u, twl[(r - 1) * 256 + j]);
          }
        }
        final_dft<LOG2N>(v, p);
        if (pilot_here && it == 0) {
          // LS estimate H = Y conj(X) / |X|^2 (1/sqrt(N) folded into xinv)
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int k = bin_of<LOG2N>(jt, e);
            h[e] = cmul(v[e], __ldg(p.xinv + k));
            if (g == 0) p.H_out[hrow + k] = h[e];
          }
          float acc[OWN];
          tmem_wait_st();
          TmE::ld(tE, acc);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 32; ++e) acc[e] = fmaf(h[e].x, h[e].x, fmaf(h[e].y, h[e].y, acc[e]));
          TmE::st(tE, acc);
        } else {
          // MRC numerator: P += conj(H) Y as four FMAs per subcarrier
          const int dl = it - (pilot_here ? 1 : 0);
          const uint32_t tp = tP + 2 * OWN * dl;
          tmem_wait_st();
#pragma unroll
          for (int q0 = 0; q0 < 64; q0 += 32) {
            float acc[32];
            Tmem<32>::ld(tp + q0, acc);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float2 hh = h[q0 / 2 + i], y = v[q0 / 2 + i];
              acc[2 * i] = fmaf(hh.x, y.x, fmaf(hh.y, y.y, acc[2 * i]));
              acc[2 * i + 1] = fmaf(hh.x, y.y, fmaf(-hh.y, y.x, acc[2 * i + 1]));
            }
            Tmem<32>::st(tp + q0, acc);
          }
        }
      }
    }
    tmem_wait_st();
    // ---- group end: every pair's steps are done, every copy of the group
    // has landed; the per-pair regions are free for the reduction
    __syncthreads();
    if (g == 0) {
      float* RE = reinterpret_cast<float*>(smem + lay.pair_off);   // [pairs][N]
      float e[OWN];
      TmE::ld(tE, e);
      tmem_wait_ld();
#pragma unroll
      for (int cc = 0; cc < OWN; ++cc) RE[q * N + bin_of<LOG2N>(jt, cc)] = e[cc];
      __syncthreads();
      for (int k = tid; k < N; k += kPThreads) {
        float E = 0.f;
#pragma unroll
        for (int w = 0; w < kPPairs; ++w) E += RE[w * N + k];
        if (p.mode == kModePartial) {
          p.E_out[(static_cast<size_t>(blockIdx.y) * gridDim.x + f) * N + k] = E;
        } else {
          // zero or non-finite energy flags the frame; z = 0 there
          const bool ok = (E > 0.f) && (E <= 3.4028234663852886e38f);
          if (!ok) latch(p.status, kStDevice);
          ie_s[k] = ok ? (1.0f / E) * p.inv_sqrtN : 0.f;
        }
      }
      __syncthreads();
    }
    float2* RP = reinterpret_cast<float2*>(smem + lay.pair_off);   // [pairs][dlc][N]
    const int dlc = min(nd, lay.pair_bytes / (N * 8));
    for (int dl0 = 0; dl0 < nd; dl0 += dlc) {
      const int n = min(dlc, nd - dl0);
      for (int j = 0; j < n; ++j) {
        float acc[2 * OWN];
        TmP::ld(tP + 2 * OWN * (dl0 + j), acc);
        tmem_wait_ld();
        float2* dst = RP + static_cast<size_t>(q * dlc + j) * N;
#pragma unroll
        for (int cc = 0; cc < OWN; ++cc)
          dst[bin_of<LOG2N>(jt, cc)] = make_float2(acc[2 * cc], acc[2 * cc + 1]);
      }
      __syncthreads();
      for (int idx = tid; idx < n * N; idx += kPThreads) {
        const int j = idx >> LOG2N;
        const int k = idx & (N - 1);
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < kPPairs; ++w) s = cadd(s, RP[static_cast<size_t>(w * dlc + j) * N + k]);
        const int dl = dl0 + j;
        if (p.mode == kModePartial) {
          p.P_out[((static_cast<size_t>(blockIdx.y) * gridDim.x + f) * p.D + d0 + dl) * N + k] =
              make_float2(s.x * p.inv_sqrtN, s.y * p.inv_sqrtN);
        } else {
          const float ie = ie_s[k];
          const float2 z = (ie != 0.f) ? make_float2(s.x * ie, s.y * ie) : make_float2(0.f, 0.f);
          if (p.eq) p.eq[(static_cast<size_t>(f) * p.D + d0 + dl) * N + k] = z;
          uint32_t code = gray(axis_level(z.x, p));
          if (p.axes == 2) code = (code << p.wbits) | gray(axis_level(z.y, p));
          codes[dl * N + k] = static_cast<uint8_t>(code);
        }
      }
      __syncthreads();
    }
    if (p.mode != kModePartial) {
      // pack: 8 consecutive subcarriers -> q bytes
      const int items8 = nd * (N / 8);
      const size_t frame_bytes = static_cast<size_t>(p.D) * N * p.q / 8;
      for (int it = tid; it < items8; it += kPThreads) {
        const int dl = it / (N / 8);
        const int k0 = (it % (N / 8)) * 8;
        uint64_t acc = 0;
#pragma unroll
        for (int bb = 0; bb < 8; ++bb) acc = (acc << p.q) | codes[dl * N + k0 + bb];
        uint8_t* dst = p.bits + f * frame_bytes + (static_cast<size_t>(d0 + dl) * N + k0) * p.q / 8;
        for (int jb = 0; jb < p.q; ++jb) dst[jb] = static_cast<uint8_t>(acc >> (8 * (p.q - 1 - jb)));
      }
      __syncthreads();   // codes consumed before the next group writes them
    }
  }
  if (issuer && p.use_tma && *abort_flag) {
    // a wait gave up: give any copy of this pair still in flight a bounded
    // chance to land before the block's shared memory is released (copies
    // stop being issued after the abort: only the issued steps count)
    for (int s = 0; s < K && s < issued; ++s) {
      const int last = issued - 1 - ((issued - 1 - s) % K);
      (void)mbar_wait_bounded(smem_u32(&bars[last % K]), (last / K) & 1);
    }
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(*tmem_base, kWTmemCols);
}

#endif  // __CUDACC__

}  // namespace lsas
