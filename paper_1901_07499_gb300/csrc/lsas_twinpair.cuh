// lsas_twinpair.cuh -- fused receiver for N = 2048 from sc16 rows: pairs of
// warps as pipelines that transform two OFDM symbols of one antenna per step,
// in split real / imaginary form.
//
// One block per frame, four pairs of warps; pair q walks antennas q, q + 4,
// ... with its own staging ring (bulk copies of the CP-stripped rows: the CP
// removal of Sec. II-B done as addressing).  A thread of a pair holds 32
// points of two symbols, the real parts of point r of both in one packed
// register pair and the imaginary parts in another, so every packed FP32
// instruction serves both symbols.  Per step (Stockham radix 32 x 8 x 8, the
// batched FFT of Sec. II-C):
//   * wait for the slot, convert both rows (exact offset floats), radix-32
//     pass by split radix (the offset leaves where two raw samples are first
//     added);
//   * middle exchange: one round of 16-byte stores {Re a, Re b, Im a, Im b},
//     half of it in the slot just read and half in the pair's exchange
//     region; pass twiddles W_2048^(8 j r) and four radix-8 DFTs;
//   * final exchange in the same two places, pass twiddles W_2048^(j r) and
//     four radix-8 DFTs;
//   * pilot: LS estimate H = Y conj(X) / |X|^2 (Sec. II-C), written out and
//     kept in registers, |H|^2 added to the channel energy (Sec. III); data
//     symbols: P += conj(H) Y in tensor memory (MRC, Sec. II-C), for two data
//     symbols as four packed FMAs per subcarrier on interleaved columns.
// Three barriers of the pair's 64 threads order a step: the first follows
// the reads of the step's slot and (in program order) every read of the
// previous step, so it also frees the previous step's slot, which is
// refilled there for the step after this one; then middle write -> read and
// final write -> read.  Middle read -> final write needs only the warp's own
// order: each warp writes its final-exchange outputs over the cells that it
// alone read in the middle exchange.
// Data-symbol groups as in the N = 1024 two-symbol kernel (the pilot with
// three data symbols, then four); at a group's end warp w < 4 adds the sums
// of warp w + 4 (same lane quarter, same subcarriers) in tensor memory, the
// two halves meet in order through shared memory, and the block forms
// z = P / E and demaps (Sec. II-B), or writes its partial sums (antenna
// split).
#pragma once

#include <type_traits>

#include "lsas_kernels.cuh"
#include "lsas_warp.cuh"
#include "lsas_twin.cuh"

namespace lsas {

constexpr int kTpPairs = 4;                  // warp pairs per block
constexpr int kTpThreads = 64 * kTpPairs;
constexpr int kTpN = 2048;
constexpr int kTpRow = kTpN * 4;             // one CP-stripped sc16 row
// middle exchange: element n = jw * 32 + rw (writer thread jw, its output
// rw) at row rw, column jw of [32][65] 16-byte entries (one pad per row);
// rows 0..15 in the slot just read, rows 16..31 in the exchange region
constexpr int kTpMRow = 65 * 16;
// final exchange: element (a, r, b) of writer j = 32 a + b (a = w + 2 i for
// warp w of the pair), output r, in the middle layout at row
// (8 i + r) ^ (bit 2 of b), column 2 b + w: the cells warp w itself read in
// the middle exchange (column parity w), without bank conflicts
constexpr int kTpSlotB = 16 * kTpMRow;       // 16,640 B: two rows, or half an exchange
constexpr int kTpTwl = 7 * 256;              // last-pass twiddles W_2048^(j r), r = 1..7

// Shared memory: header (mbarriers [pair][kMaxSlots], TMEM address, flags),
// the last-pass twiddles as {wr, wi} at [(r - 1) * 256 + j], the middle-pass
// twiddles W_2048^(8 b r) at [(r - 1) * 32 + b] (contiguous for the lanes of
// a warp), 1/E per subcarrier, then per pair: two staging slots and the
// exchange region.  At group ends the pair regions hold the partial sums
// ([2][4][N] complex) and, after them, the demapped codes of the group.
struct TpLayout {
  int tw_off, mtw_off, ie_off, codes_off, pair_off, stage_bytes, pair_bytes, total;
};
__host__ __device__ inline TpLayout make_tplayout() {
  TpLayout l;
  l.tw_off = kWHeader;
  l.mtw_off = l.tw_off + kTpTwl * 8;
  l.ie_off = l.mtw_off + 7 * 32 * 8;
  l.pair_off = align_up(l.ie_off + kTpN * 4, 128);
  l.stage_bytes = 2 * kTpSlotB;
  l.pair_bytes = align_up(l.stage_bytes + kTpSlotB, 128);
  l.codes_off = l.pair_off + 2 * kTwDg * kTpN * 8;
  l.total = l.pair_off + kTpPairs * l.pair_bytes;
  return l;
}

#ifdef __CUDACC__

// Copies of one step into a slot: items ia and ia + 1 of a group (the
// second may be absent); thread 0 registers the bytes and copies row a,
// thread 1 copies row b.
__device__ __forceinline__ void tp_issue(const KParams& p, int f, int m, bool pilot_here, int d0,
                                         int items, int ia, unsigned char* slot, uint32_t bar,
                                         uint64_t pol, int jt) {
  if (jt < 2 && ia + jt < items) {
    if (jt == 0) mbar_expect_tx(bar, ia + 1 < items ? 2 * kTpRow : kTpRow);
    bulk_load(smem_u32(slot + jt * kTpRow),
              row_ptr<11, false>(p, f, m, witem_symbol(p, pilot_here, d0, ia + jt)), kTpRow,
              bar, pol);
  }
}

// Four radix-8 DFTs of both symbols on register groups i * 8 .. i * 8 + 7
// (split radix, natural order in and out).
__device__ __forceinline__ void tp_dft8x4(float2 (&re)[32], float2 (&im)[32]) {
  Cx2 out[32];
  twin_sr<8, 0, 1, 0, false>(re, im, out);
  twin_sr<8, 8, 1, 8, false>(re, im, out);
  twin_sr<8, 16, 1, 16, false>(re, im, out);
  twin_sr<8, 24, 1, 24, false>(re, im, out);
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    re[i] = out[i].re;
    im[i] = out[i].im;
  }
}

// x * w for a pair of points and a twiddle {wr, wi} (broadcast operands)
__device__ __forceinline__ void tp_twiddle(float2& xr, float2& xi, float2 w) {
  const float2 r = __ffma2_rn(xi, f2(-w.y), __fmul2_rn(xr, f2(w.x)));
  const float2 i = __ffma2_rn(xr, f2(w.y), __fmul2_rn(xi, f2(w.x)));
  xr = r;
  xi = i;
}

template <int LOG2N>
__global__ void __launch_bounds__(kTpThreads, 1) twinpair_kernel(const KParams p) {
  static_assert(LOG2N == 11, "the two-symbol pair kernel is written for N = 2048");
  constexpr int N = 1 << LOG2N;
  constexpr int OWN = kTwOwn;
  constexpr int K = 2;
  using TmE = Tmem<OWN>;
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int q = warp >> 1;          // pair
  const int jt = tid & 63;          // FFT team thread
  const int pbar = 1 + q;           // the pair's named barrier (0 is the block's)
  const TpLayout lay = make_tplayout();
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem) + q * kMaxSlots;
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(smem + kWTmemAddr);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kWAbort);
  float2* twl = reinterpret_cast<float2*>(smem + lay.tw_off);   // [r - 1][j]
  float2* mtw = reinterpret_cast<float2*>(smem + lay.mtw_off);  // [r - 1][b]
  float* ie_s = reinterpret_cast<float*>(smem + lay.ie_off);
  uint8_t* codes = smem + lay.codes_off;
  unsigned char* stage = smem + lay.pair_off + q * lay.pair_bytes;
  unsigned char* const X = stage + lay.stage_bytes;

  for (int i = tid; i < kTpTwl; i += kTpThreads) twl[i] = __ldg(p.twP + 512 + i);
  for (int i = tid; i < 7 * 32; i += kTpThreads) mtw[i] = __ldg(p.twP + 32 + i);
  if (tid == 0) *abort_flag = 0;
  if (jt == 0) {
    for (int s = 0; s < K; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_base), kWTmemCols);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  // this warp's columns: 256 columns of its lane quarter; warp w + 4 holds
  // the same subcarriers (same jt) in the other half of the quarter
  const uint32_t tE = *tmem_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                      static_cast<uint32_t>((warp >> 2) * kTwTmemWarp);
  const uint64_t pol = jt < 2 ? evict_first_policy() : 0;
  float zero[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) zero[i] = 0.f;

  const int nch = q < p.chunks ? (p.chunks - 1 - q) / kTpPairs + 1 : 0;
  // start the pairs of the upper half a little later, so that the two warps
  // sharing a scheduler tend to be in different phases of their steps
  if (warp >= 4) __nanosleep(1400);
  int issued = 0;  // steps whose copies this pair has issued
  int slot = 0;    // ring slot of the next step to consume ...
  int phase = 0;   // ... and its mbarrier phase
  // one data-symbol group per grid z index (partial mode, small batches):
  // every group's block transforms the pilot itself; group 0 alone writes H
  // and the channel energy
  const int g_lo = p.group_z ? static_cast<int>(blockIdx.z) : 0;
  const int g_hi = p.group_z ? g_lo + 1 : twin_groups(p.D);
  for (int g = g_lo; g < g_hi; ++g) {
    const int d0 = g == 0 ? 0 : kTwDg0 + (g - 1) * kTwDg;
    const int nd = min(g == 0 ? kTwDg0 : kTwDg, p.D - d0);
    const bool pilot_here = g == 0 || p.group_z;
    const bool energy_here = g == 0;
    const int items = nd + (pilot_here ? 1 : 0);
    const int npairs = (items + 1) / 2;
    const uint32_t tP = energy_here ? tE + OWN : tE;
    if (energy_here) {
#pragma unroll
      for (int q0 = 0; q0 < OWN; q0 += 16) Tmem<16>::st(tE + q0, zero);
    }
    for (uint32_t c = tP; c < tE + kTwTmemWarp; c += 16) Tmem<16>::st(c, zero);
    // issue cursor: local chunk and pair of the next step to stage, and how
    // many steps of this group are still to be staged
    int ic = 0, ipi = 0;
    int to_issue = nch * npairs;
    if (!*abort_flag) {
      // the ring held generic data (last group's reduction): order it before
      // the copies, then fill the first K slots of this group
      fence_proxy_async();
      int is = slot;
      for (int s = 0; s < K && to_issue > 0; ++s, --to_issue) {
        tp_issue(p, f, q + ic * kTpPairs, pilot_here, d0, items, 2 * ipi, stage + is * kTpSlotB,
                 smem_u32(&bars[is]), pol, jt);
        // test hook: the first staging phase of block 0 also waits for 16
        // bytes that no copy delivers, so its bounded wait runs out
        if (p.fault == 1 && blockIdx.x == 0 && q == 0 && g == 0 && s == 0 && jt == 0)
          mbar_expect_tx_only(smem_u32(&bars[is]), 16);
        ++issued;
        is = (is + 1 == K) ? 0 : is + 1;
        if (++ipi == npairs) {
          ipi = 0;
          ++ic;
        }
      }
    }
    unsigned char* prev_slot = nullptr;   // slot of the pair's previous step in this group
    uint32_t prev_bar = 0;
    for (int lc = 0; lc < nch; ++lc) {
      const int m = q + lc * kTpPairs;
      const size_t hrow = (static_cast<size_t>(f) * p.Mtot + p.m0 + blockIdx.y * p.shard_y + m) * N;
      float2 h[32];
      if (!pilot_here) {
#pragma unroll
        for (int e = 0; e < 32; ++e) h[e] = p.H_out[hrow + bin_of<LOG2N>(jt, e)];
      }
      for (int ip = 0; ip < npairs; ++ip) {
        float2 re[32], im[32];
        wait_slot(smem_u32(&bars[slot]), phase, abort_flag, p.status);
        unsigned char* const yslot = stage + slot * kTpSlotB;
        const uint32_t ybar = smem_u32(&bars[slot]);
        {
          // both rows; a missing second row leaves earlier contents of the
          // slot (finite values), whose transform is not used
          const uint32_t* sa = reinterpret_cast<const uint32_t*>(yslot);
          const uint32_t* sb = sa + kTpRow / 4;
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            // sc16 -> float v + 2^23 + 32768 exactly: sign bits flipped to
            // offset binary, each half placed under the exponent bytes of
            // 2^23 (the offset leaves where pass 1 first adds two samples)
            const uint32_t ua = sa[jt + 64 * r] ^ 0x80008000u;
            const uint32_t ub = sb[jt + 64 * r] ^ 0x80008000u;
            re[r] = make_float2(__uint_as_float(__byte_perm(ua, 0x4b000000u, 0x7610)),
                                __uint_as_float(__byte_perm(ub, 0x4b000000u, 0x7610)));
            im[r] = make_float2(__uint_as_float(__byte_perm(ua, 0x4b000000u, 0x7632)),
                                __uint_as_float(__byte_perm(ub, 0x4b000000u, 0x7632)));
          }
        }
        if (++slot == K) {
          slot = 0;
          phase ^= 1;
        }
        // pass 1: 32-point DFTs over n1 (n = jt + 64 n1); output k1 = r
        twin_dft32_sr<true>(re, im);
        // B0: both warps have read this step's slot and finished the previous
        // step's reads: the previous slot is refilled, and this step's slot
        // and the exchange region take the middle exchange
        bar_sync(pbar, 64);
        if (prev_slot && to_issue > 0 && !*abort_flag) {
          ++issued;
          fence_proxy_async();
          tp_issue(p, f, q + ic * kTpPairs, pilot_here, d0, items, 2 * ipi, prev_slot, prev_bar, pol,
                   jt);
          --to_issue;
          if (++ipi == npairs) {
            ipi = 0;
            ++ic;
          }
        }
        prev_slot = yslot;
        prev_bar = ybar;
        // middle exchange: Y1[jt * 32 + r] at row r, column jt
#pragma unroll
        for (int r = 0; r < 32; ++r)
          *reinterpret_cast<float4*>((r < 16 ? yslot : X) + ((r & 15) * 65 + jt) * 16) =
              make_float4(re[r].x, re[r].y, im[r].x, im[r].y);
        bar_sync(pbar, 64);   // B1
        {
          // Y1[j + 256 rr], j = jt + 64 i: writer (jt >> 5) + 2 i + 8 rr, its
          // output jt & 31
          const unsigned char* mrow = ((jt & 16) ? X : yslot) + (jt & 15) * kTpMRow;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
              const float4 v = *reinterpret_cast<const float4*>(mrow + ((jt >> 5) + 2 * i + 8 * rr) * 16);
              re[i * 8 + rr] = make_float2(v.x, v.y);
              im[i * 8 + rr] = make_float2(v.z, v.w);
            }
          }
        }
        // middle-pass twiddles W_2048^(8 (jt & 31) rr)
#pragma unroll
        for (int rr = 1; rr < 8; ++rr) {
          const float2 w = mtw[(rr - 1) * 32 + (jt & 31)];
#pragma unroll
          for (int i = 0; i < 4; ++i) tp_twiddle(re[i * 8 + rr], im[i * 8 + rr], w);
        }
        tp_dft8x4(re, im);
        // final exchange: output r of j = jt + 64 i = 32 a + b (a = w + 2 i,
        // w = jt >> 5 the warp of the pair) goes to row R = (8 i + r) ^ t,
        // column 2 b + w of the middle layout (t = bit 2 of b spreads a
        // quarter-warp's 16-byte cells over all banks).  Warp w writes only
        // the column-parity-w cells that it alone read in the middle
        // exchange, so its own reads need to be done, not its partner's
        __syncwarp();
        const int tq = (jt >> 2) & 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int R = (8 * i + r) ^ tq;
            *reinterpret_cast<float4*>((i < 2 ? yslot : X) + ((R & 15) * 65 + 2 * (jt & 31) + (jt >> 5)) * 16) =
                make_float4(re[i * 8 + r].x, re[i * 8 + r].y, im[i * 8 + r].x, im[i * 8 + r].y);
          }
        }
        bar_sync(pbar, 64);   // B2
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int a = (jt >> 5) + 2 * i;   // this thread's j = jt + 64 i = 32 a + (jt & 31)
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            // output a of j' = 32 r + b, written by warp r & 1 at its i' = r >> 1
            const int R = (8 * (r >> 1) + a) ^ tq;
            const float4 v = *reinterpret_cast<const float4*>(
                (r < 4 ? yslot : X) + ((R & 15) * 65 + 2 * (jt & 31) + (r & 1)) * 16);
            re[i * 8 + r] = make_float2(v.x, v.y);
            im[i * 8 + r] = make_float2(v.z, v.w);
            if (r > 0) tp_twiddle(re[i * 8 + r], im[i * 8 + r], twl[(r - 1) * 256 + jt + 64 * i]);
          }
        }
        // last pass: register e holds bin bin_of(jt, e)
        tp_dft8x4(re, im);
        const int ia = 2 * ip;
        if (pilot_here && ip == 0) {
          // first row: the pilot.  LS estimate H = Y conj(X) / |X|^2 (1/sqrt(N)
          // folded into xinv); group 0 writes it out and adds |H|^2 into the
          // energy
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int k = bin_of<LOG2N>(jt, e);
            const float2 hv = cmul(make_float2(re[e].x, im[e].x), __ldg(p.xinv + k));
            h[e] = hv;
            if (energy_here) p.H_out[hrow + k] = hv;
          }
          if (energy_here) {
            float acc[OWN];
            tmem_wait_st();
            TmE::ld(tE, acc);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 32; ++e) acc[e] = fmaf(h[e].x, h[e].x, fmaf(h[e].y, h[e].y, acc[e]));
            TmE::st(tE, acc);
          }
          bool pr;
          if (1 < items) twin_mrc<1>(re, im, h, tP + twin_block_col(1, true, &pr, items));
        } else {
          bool pr;
          const uint32_t tb = tP + twin_block_col(ia, pilot_here, &pr, items);
          if (pr) {
            twin_mrc2(re, im, h, tb);
          } else {
            twin_mrc<0>(re, im, h, tb);
          }
        }
      }
    }
    tmem_wait_st();
    // ---- group end: every pair's steps are done and every copy of the
    // group has landed; the pair regions are free for the reduction, and the
    // tensor-memory stores of every warp are ordered before the loads of its
    // lane-quarter partner
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (energy_here) {
      // warp w < 4 (pairs 0, 1) adds warp w + 4's columns (pairs 2, 3)
      float* RE = reinterpret_cast<float*>(smem + lay.pair_off);   // [2][N]
      if (warp < 4) {
        float e[OWN], e2[OWN];
        TmE::ld(tE, e);
        TmE::ld(tE + kTwTmemWarp, e2);
        tmem_wait_ld();
#pragma unroll
        for (int cc = 0; cc < OWN; ++cc) RE[q * N + bin_of<LOG2N>(jt, cc)] = e[cc] + e2[cc];
      }
      __syncthreads();
      for (int k = threadIdx.x; k < N; k += kTpThreads) {
        const float E = RE[k] + RE[N + k];
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
    {
      // the group's data items in tensor memory, block by block (a step's
      // pair of items interleaved in 128 columns, or an item alone in 64):
      // the two warps of a lane quarter (pairs q and q + 2) take alternate
      // blocks, add both warps' sums and write them to shared memory
      float2* RP = reinterpret_cast<float2*>(smem + lay.pair_off);   // [2][kTwDg][N]
      const uint32_t tfirst = tE - static_cast<uint32_t>((warp >> 2) * kTwTmemWarp);   // first warp's columns
      const int j0 = pilot_here ? 1 : 0;
      int blk = 0;
      for (int it = j0; it < items; ++blk) {
        bool pr;
        const uint32_t tb = tfirst + (tP - tE) + twin_block_col(it, pilot_here, &pr, items);
        if ((blk & 1) == (warp >> 2)) {
          float2* dst = RP + static_cast<size_t>((q & 1) * kTwDg + (it - j0)) * N;
          if (pr) {
#pragma unroll
            for (int q0 = 0; q0 < 128; q0 += 32) {
              float t[32], t2[32];
              Tmem<32>::ld(tb + q0, t);
              Tmem<32>::ld(tb + kTwTmemWarp + q0, t2);
              tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int k = bin_of<LOG2N>(jt, q0 / 4 + i);
                dst[k] = make_float2(t[4 * i] + t2[4 * i], t[4 * i + 2] + t2[4 * i + 2]);
                dst[N + k] = make_float2(t[4 * i + 1] + t2[4 * i + 1], t[4 * i + 3] + t2[4 * i + 3]);
              }
            }
          } else {
#pragma unroll
            for (int q0 = 0; q0 < 2 * OWN; q0 += 32) {
              float t[32], t2[32];
              Tmem<32>::ld(tb + q0, t);
              Tmem<32>::ld(tb + kTwTmemWarp + q0, t2);
              tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < 16; ++i)
                dst[bin_of<LOG2N>(jt, q0 / 2 + i)] =
                    make_float2(t[2 * i] + t2[2 * i], t[2 * i + 1] + t2[2 * i + 1]);
            }
          }
        }
        it += pr ? 2 : 1;
      }
      __syncthreads();
      // eight items per thread at a time: their shared-memory sums are all
      // loaded before the first is demapped; one copy of the loop per
      // constellation, so that the slicer inside it has no branches
      auto demap_items = [&](auto tcount) {
        constexpr int T = decltype(tcount)::value;
        for (int idx0 = threadIdx.x; idx0 < nd * N; idx0 += 8 * kTpThreads) {
          float2 sv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int idx = min(idx0 + u * kTpThreads, nd * N - 1);
            const int dl = idx >> LOG2N;
            const int k = idx & (N - 1);
            sv[u] = cadd(RP[static_cast<size_t>(dl) * N + k], RP[static_cast<size_t>(kTwDg + dl) * N + k]);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int idx = idx0 + u * kTpThreads;
            if (idx >= nd * N) break;
            const int dl = idx >> LOG2N;
            const int k = idx & (N - 1);
            const float2 s = sv[u];
            if (p.mode == kModePartial) {
              p.P_out[((static_cast<size_t>(blockIdx.y) * gridDim.x + f) * p.D + d0 + dl) * N + k] =
                  make_float2(s.x * p.inv_sqrtN, s.y * p.inv_sqrtN);
            } else {
              const float ie = ie_s[k];
              const float2 z = (ie != 0.f) ? make_float2(s.x * ie, s.y * ie) : make_float2(0.f, 0.f);
              if (p.eq) p.eq[(static_cast<size_t>(f) * p.D + d0 + dl) * N + k] = z;
              uint32_t code = gray(count_ge<T>(z.x, p.thr));
              if (p.axes == 2) code = (code << p.wbits) | gray(count_ge<T>(z.y, p.thr));
              codes[dl * N + k] = static_cast<uint8_t>(code);
            }
          }
        }
      };
      switch (p.nthr) {
        case 1: demap_items(std::integral_constant<int, 1>{}); break;
        case 3: demap_items(std::integral_constant<int, 3>{}); break;
        case 7: demap_items(std::integral_constant<int, 7>{}); break;
        default: demap_items(std::integral_constant<int, kMaxThresholds>{}); break;
      }
      __syncthreads();
    }
    if (p.mode != kModePartial) {
      // pack: 8 consecutive subcarriers -> q bytes
      const int items8 = nd * (N / 8);
      const size_t frame_bytes = static_cast<size_t>(p.D) * N * p.q / 8;
      for (int it = threadIdx.x; it < items8; it += kTpThreads) {
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
  if (jt == 0 && *abort_flag) {
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
