// lsas_twin.cuh -- fused receiver for N = 256 .. 1024 from sc16 rows, two
// OFDM symbols per warp step, in split real / imaginary form.
//
// One block per frame, 8 warps, each an independent pipeline over antenna
// rows, as in the per-warp kernel.  At N = 1024 a warp step takes one
// antenna (warp w takes antennas w, w + 8, ...); for smaller N the warp's
// lanes form A = 1024 / N teams of L = N / 32 lanes, team t taking antenna
// (w + 8 c) A + t at the warp's step c, so every step still moves 32 points
// per lane.  What differs from the per-warp kernel is the unit of a step: a
// lane holds 32 points of TWO symbols of its antenna, the real parts of
// point r of both symbols in one packed
// register pair and the imaginary parts in another.  Every packed FP32
// instruction then applies one operation to both symbols: a product by a
// twiddle takes four packed instructions for two points and no operand
// rearrangement, a product by -j is a renaming, and each warp has two
// independent transforms in flight.  The antenna's channel, held in
// registers, serves both symbols of a step.
//
// Per step a warp
//   * waits for its staging slot (bulk copies of the two CP-stripped rows:
//     the CP removal of Sec. II-B done as addressing),
//   * runs the radix-32 pass (the batched FFT of Sec. II-C) in registers,
//     transposes through the slot it has just read and its own exchange
//     region, refills the slot, applies the pass twiddles and runs the
//     second radix-32 pass,
//   * pilot: LS estimate H = Y conj(X) / |X|^2 (Sec. II-C), written out and
//     kept in registers, and |H|^2 added to the channel energy (Sec. III);
//     data symbol: P += conj(H) Y per subcarrier in the warp's tensor-memory
//     columns (the MRC numerator, Sec. II-C); for two data symbols as four
//     packed FMAs per subcarrier on their interleaved columns.
// The second pass is radix L: it reads column jt of the exchange (32 rows of
// L points per team) and takes 32 / L DFTs of L points per symbol.
// Data-symbol groups: the pilot with the first three data symbols, then four
// data symbols at a time (a warp's 256 TMEM columns hold the energy and three
// symbols' sums, or four symbols' sums), so the 14 rows of a frame with 13
// data symbols pair up exactly.  Each lane keeps 32 subcarriers of its own
// antenna whatever N is, so the grouping is the same for every N; that is
// why the one-symbol kernel (which sums a step's antennas across lanes and
// needs one group at N = 256) stays the choice for few antennas per launch.  At a group's end each warp w < 4 adds the
// sums of warp w + 4 (its lane-quarter partner) in tensor memory, the four
// results meet in warp order through shared memory, and the block forms
// z = P / E and demaps (Sec. II-B), or writes its partial sums (antenna
// split).
#pragma once

#include <type_traits>

#include "lsas_kernels.cuh"
#include "lsas_warp.cuh"

namespace lsas {

constexpr int kTwWarps = 8;
constexpr int kTwThreads = 32 * kTwWarps;
constexpr int kTwSlots = 2;                 // staging slots per warp, two rows each
constexpr int kTwTmemWarp = 256;            // TMEM columns per warp
constexpr int kTwOwn = 32;                  // subcarriers per lane
constexpr int kTwDg0 = (kTwTmemWarp - kTwOwn) / (2 * kTwOwn);   // 3: group 0
constexpr int kTwDg = kTwTmemWarp / (2 * kTwOwn);                // 4: later groups
// The exchange between the passes is one round of 16-byte stores of
// {Re a, Re b, Im a, Im b} per point: row n2 (32 points, 528 bytes with a
// 16-byte pad, so that both the row stores and the column loads are free of
// bank conflicts) goes to the slot just read for n2 < 16 and to the warp's
// exchange region for n2 >= 16.
constexpr int kTwXRow = 32 * 16 + 16;       // one padded exchange row
constexpr int kTwSlotB = 16 * kTwXRow;      // a slot: two sc16 rows, or 16 exchange rows
constexpr int kTwXS = 16 * kTwXRow / 8;     // exchange region (float2): the other 16 rows
// A slot holds the step's rows as two halves (the two symbols) of 1056 words:
// the A = 32 / L antennas of a warp step (L = N / 32 lanes each) at N + L
// words apart, so that the lanes' loads of a row position hit distinct banks.
constexpr int kTwHalfB = 32 * 33 * 4;

// Shared memory: header (mbarriers, TMEM address, flags), the pass twiddles
// W_N^(j r) as {wr, wi} at [r * 32 + j] (N entries), 1/E per subcarrier, the
// demapped codes of one group, then one region per warp: its staging ring
// (two slots) and its exchange region.  At group ends the per-warp regions together hold
// the warps' partial sums for the cross-warp reduction.
struct TwLayout {
  int tw_off, ie_off, codes_off, warp_off, stage_bytes, warp_bytes, total;
};
__host__ __device__ inline TwLayout make_twlayout() {
  TwLayout l;
  l.tw_off = kWHeader;
  l.ie_off = l.tw_off + 1024 * 8;
  l.codes_off = l.ie_off + 1024 * 4;
  l.warp_off = align_up(l.codes_off + kTwDg * 1024, 128);
  l.stage_bytes = kTwSlots * kTwSlotB;
  l.warp_bytes = align_up(l.stage_bytes + kTwXS * 8, 128);
  l.total = l.warp_off + kTwWarps * l.warp_bytes;
  return l;
}
// data-symbol groups of a frame with D data symbols
__host__ __device__ inline int twin_groups(int D) {
  const int rest = D > kTwDg0 ? D - kTwDg0 : 0;
  return 1 + (rest + kTwDg - 1) / kTwDg;
}

#ifdef __CUDACC__

// Two complex values, one per symbol of a step: re = {Re a, Re b},
// im = {Im a, Im b}.
struct Cx2 {
  float2 re, im;
};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// cos(2 pi e / 32) for a compile-time e, from the first octant: kC[e] =
// cos(2 pi e / 32) to double precision, rounded once to float.
__device__ __forceinline__ float twin_cos32(int e) {
  constexpr float kC[9] = {1.0f,
                           0.98078528040323043f, 0.92387953251128674f,
                           0.83146961230254524f, 0.70710678118654757f,
                           0.55557023301960229f, 0.38268343236508984f,
                           0.19509032201612833f, 0.0f};
  e &= 31;
  return e <= 8 ? kC[e] : e <= 16 ? -kC[16 - e] : e <= 24 ? -kC[e - 16] : kC[32 - e];
}

// W_32^e z for a compile-time e: W = {c, -s}, W z = {Re z c + Im z s,
// Im z c - Re z s}, four packed instructions.
__device__ __forceinline__ Cx2 twin_wmul(const Cx2& z, int e) {
  const float c = twin_cos32(e), s = twin_cos32(8 - e);
  return {__ffma2_rn(z.im, f2(s), __fmul2_rn(z.re, f2(c))),
          __ffma2_rn(z.re, f2(-s), __fmul2_rn(z.im, f2(c)))};
}

// The split-radix step of an N-point DFT (Sec. II-C's FFT, split radix):
// with U the N/2-point DFT of the even samples and Z, Z' the N/4-point DFTs
// of samples 4n + 1 and 4n + 3, for k < N/4 and a = W_N^k Z[k],
// b = W_N^3k Z'[k]:  X[k] = U[k] + (a + b), X[k + N/2] = U[k] - (a + b),
// X[k + N/4] = U[k + N/4] - j (a - b), X[k + 3N/4] = U[k + N/4] + j (a - b),
// in place on x0..x3 = U[k], U[k + N/4], Z[k], Z'[k].  OFS: Z and Z' are raw
// samples carrying the offset c (N = 4), removed from their sum.
template <int N, bool OFS>
__device__ __forceinline__ void twin_lbfly(Cx2& x0, Cx2& x1, Cx2& x2, Cx2& x3, int k) {
  constexpr float kS = 0.70710678118654752440f;   // 1/sqrt(2)
  const int e = k * (32 / N);                      // W_N^k = W_32^e
  const Cx2 U = x0, U2 = x1, Z = x2, Z2 = x3;
  if (e == 4) {
    // W_8 and W_8^3: a = s {Re Z + Im Z, Im Z - Re Z}, b = s {u, -t} with
    // u = Im Z' - Re Z', t = Re Z' + Im Z'; the scale s = 1/sqrt2 enters the sums
    const float2 ar = cadd(Z.re, Z.im), ai = csub(Z.im, Z.re);
    const float2 u = csub(Z2.im, Z2.re), t = cadd(Z2.re, Z2.im);
    const float2 sr = cadd(ar, u), si = csub(ai, t), dr = csub(ar, u), di = cadd(ai, t);
    x0 = {__ffma2_rn(sr, f2(kS), U.re), __ffma2_rn(si, f2(kS), U.im)};
    x2 = {__ffma2_rn(sr, f2(-kS), U.re), __ffma2_rn(si, f2(-kS), U.im)};
    x1 = {__ffma2_rn(di, f2(kS), U2.re), __ffma2_rn(dr, f2(-kS), U2.im)};
    x3 = {__ffma2_rn(di, f2(-kS), U2.re), __ffma2_rn(dr, f2(kS), U2.im)};
    return;
  }
  Cx2 s, d;
  if (k == 0) {
    const Cx2 b = OFS ? Cx2{cadd(Z2.re, f2(-16842752.0f)), cadd(Z2.im, f2(-16842752.0f))} : Z2;
    s = {cadd(Z.re, b.re), cadd(Z.im, b.im)};
    d = {csub(Z.re, Z2.re), csub(Z.im, Z2.im)};
  } else {
    const Cx2 a = twin_wmul(Z, e), b = twin_wmul(Z2, 3 * e);
    s = {cadd(a.re, b.re), cadd(a.im, b.im)};
    d = {csub(a.re, b.re), csub(a.im, b.im)};
  }
  x0 = {cadd(U.re, s.re), cadd(U.im, s.im)};
  x2 = {csub(U.re, s.re), csub(U.im, s.im)};
  x1 = {cadd(U2.re, d.im), csub(U2.im, d.re)};
  x3 = {csub(U2.re, d.im), cadd(U2.im, d.re)};
}

// X[B + k], k < N: the N-point DFT of the samples re/im[O + S n], n < N,
// by split radix (recursion at compile time).  OFS: the samples carry the
// offset c = 2^23 + 32768 on each part, removed exactly where two raw
// samples are first added (a + (b - 2c)); their differences are exact.
template <int N, int O, int S, int B, bool OFS>
__device__ __forceinline__ void twin_sr(const float2 (&re)[32], const float2 (&im)[32],
                                        Cx2 (&out)[32]) {
  if constexpr (N == 1) {
    out[B] = {re[O], im[O]};
  } else if constexpr (N == 2) {
    const Cx2 a = {re[O], im[O]}, b = {re[O + S], im[O + S]};
    if constexpr (OFS) {
      out[B] = {cadd(a.re, cadd(b.re, f2(-16842752.0f))), cadd(a.im, cadd(b.im, f2(-16842752.0f)))};
    } else {
      out[B] = {cadd(a.re, b.re), cadd(a.im, b.im)};
    }
    out[B + 1] = {csub(a.re, b.re), csub(a.im, b.im)};
  } else {
    twin_sr<N / 2, O, 2 * S, B, OFS>(re, im, out);
    twin_sr<N / 4, O + S, 4 * S, B + N / 2, OFS>(re, im, out);
    twin_sr<N / 4, O + 3 * S, 4 * S, B + 3 * N / 4, OFS>(re, im, out);
#pragma unroll
    for (int k = 0; k < N / 4; ++k)
      twin_lbfly<N, OFS && N == 4>(out[B + k], out[B + N / 4 + k], out[B + N / 2 + k],
                                   out[B + 3 * N / 4 + k], k);
  }
}

template <bool OFS>
__device__ __forceinline__ void twin_dft32_sr(float2 (&re)[32], float2 (&im)[32]) {
  Cx2 out[32];
  twin_sr<32, 0, 1, 0, OFS>(re, im, out);
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    re[i] = out[i].re;
    im[i] = out[i].im;
  }
}

// Pass 2: the 32 / L radix-L DFTs of both symbols on register groups
// i L .. i L + L - 1 (split radix, natural order in and out).
template <int L>
__device__ __forceinline__ void twin_pass2(float2 (&re)[32], float2 (&im)[32]) {
  if constexpr (L == 32) {
    twin_dft32_sr<false>(re, im);
  } else {
    Cx2 out[32];
    twin_sr<L, 0, 1, 0, false>(re, im, out);
    twin_sr<L, L, 1, L, false>(re, im, out);
    if constexpr (L <= 8) {
      twin_sr<L, 2 * L, 1, 2 * L, false>(re, im, out);
      twin_sr<L, 3 * L, 1, 3 * L, false>(re, im, out);
    }
    if constexpr (L <= 4) {
      twin_sr<L, 4 * L, 1, 4 * L, false>(re, im, out);
      twin_sr<L, 5 * L, 1, 5 * L, false>(re, im, out);
      twin_sr<L, 6 * L, 1, 6 * L, false>(re, im, out);
      twin_sr<L, 7 * L, 1, 7 * L, false>(re, im, out);
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      re[i] = out[i].re;
      im[i] = out[i].im;
    }
  }
}

// Issue the bulk copies of one step: items ia and ia + 1 of a group (the
// second may be absent) for the A antennas of chunk c.  Lane h A + t copies
// the row of symbol item ia + h of antenna c A + t to half h of the slot,
// team t's place (rows L words apart, for conflict-free loads); lane 0
// registers the bytes.
template <int LOG2N>
__device__ __forceinline__ void twin_issue(const KParams& p, int f, int c, bool pilot_here, int d0,
                                           int items, int ia, unsigned char* slot, uint32_t bar,
                                           uint64_t pol, int lane) {
  constexpr int N = 1 << LOG2N, L = N / 32, A = 32 / L;
  constexpr uint32_t bytes = N * 4;
  const int nant = min(A, p.M - c * A);
  const int nrow = ia + 1 < items ? 2 : 1;
  if (lane == 0) mbar_expect_tx(bar, bytes * nant * nrow);
  if (lane < 2 * A) {
    const int half = lane / A, t = lane % A;
    if (t < nant && half < nrow)
      bulk_load(smem_u32(slot + half * kTwHalfB + t * (N + L) * 4),
                row_ptr<LOG2N, false>(p, f, c * A + t, witem_symbol(p, pilot_here, d0, ia + half)),
                bytes, bar, pol);
  }
}

// P += conj(H) Y for one symbol of the step (half 0: .x, half 1: .y) into
// the 64 accumulator columns at tp (columns 2c, 2c + 1 for the subcarrier of
// register c), as four FMAs per subcarrier.
template <int HALF, int QC = 16>
__device__ __forceinline__ void twin_mrc(const float2 (&re)[32], const float2 (&im)[32],
                                         const float2 (&h)[32], uint32_t tp) {
  tmem_wait_st();
#pragma unroll
  for (int q0 = 0; q0 < 64; q0 += QC) {
    float acc[QC];
    Tmem<QC>::ld(tp + q0, acc);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < QC / 2; ++i) {
      const int e = q0 / 2 + i;
      const float2 hh = h[e];
      const float yr = HALF ? re[e].y : re[e].x;
      const float yi = HALF ? im[e].y : im[e].x;
      acc[2 * i] = fmaf(hh.x, yr, fmaf(hh.y, yi, acc[2 * i]));
      acc[2 * i + 1] = fmaf(hh.x, yi, fmaf(-hh.y, yr, acc[2 * i + 1]));
    }
    Tmem<QC>::st(tp + q0, acc);
  }
}

// P += conj(H) Y for both symbols of a step into the 128 interleaved
// columns at tp (4c: Re a, 4c + 1: Re b, 4c + 2: Im a, 4c + 3: Im b for
// the subcarrier of register c): the symbols' values are already packed pairs, so
// four packed FMAs per subcarrier, in the scalar form's order of operations.
__device__ __forceinline__ void twin_mrc2(const float2 (&re)[32], const float2 (&im)[32],
                                          const float2 (&h)[32], uint32_t tp) {
  tmem_wait_st();
#pragma unroll
  for (int q0 = 0; q0 < 128; q0 += 32) {
    float acc[32];
    Tmem<32>::ld(tp + q0, acc);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = q0 / 4 + i;
      const float2 hr = f2(h[e].x), hi = f2(h[e].y), nhi = f2(-h[e].y);
      const float2 pr = __ffma2_rn(hr, re[e], __ffma2_rn(hi, im[e], make_float2(acc[4 * i], acc[4 * i + 1])));
      const float2 pi = __ffma2_rn(hr, im[e], __ffma2_rn(nhi, re[e], make_float2(acc[4 * i + 2], acc[4 * i + 3])));
      acc[4 * i] = pr.x;
      acc[4 * i + 1] = pr.y;
      acc[4 * i + 2] = pi.x;
      acc[4 * i + 3] = pi.y;
    }
    Tmem<32>::st(tp + q0, acc);
  }
}

// Accumulator columns of item `it` of a group (data items only; the pilot,
// when the group transforms it, is item 0), relative to the group's first
// partial-sum column: a step whose two items are both data symbols keeps
// them interleaved in 128 columns (twin_mrc2), a data item alone in its step
// (beside the pilot, or last of an odd count) 64 columns (2c: Re, 2c + 1: Im).
__device__ __forceinline__ int twin_block_col(int it, bool pilot, bool* pair, int items) {
  const int ip = it >> 1;
  *pair = !(pilot && ip == 0) && (2 * ip + 1 < items);
  return pilot ? (ip == 0 ? 0 : 64 + 128 * (ip - 1)) : 128 * ip;
}

template <int LOG2N>
__global__ void __launch_bounds__(kTwThreads, 1) twin_kernel(const KParams p) {
  static_assert(LOG2N >= 7 && LOG2N <= 10, "the two-symbol kernel covers N = 128 .. 1024");
  constexpr int N = 1 << LOG2N;
  constexpr int L = N / 32;     // lanes of an antenna's FFT team
  constexpr int A = 32 / L;     // antennas of a warp step (teams)
  constexpr int NW = kTwWarps;
  constexpr int NT = kTwThreads;
  constexpr int OWN = kTwOwn;
  constexpr int K = kTwSlots;
  using TmP = Tmem<2 * OWN>;   // one data symbol of partial sums (complex)
  using TmE = Tmem<OWN>;       // channel energy
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int team = lane / L;    // antenna of the chunk
  const int jt = lane % L;      // FFT team thread
  const TwLayout lay = make_twlayout();
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem) + warp * kMaxSlots;
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(smem + kWTmemAddr);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kWAbort);
  float2* tws = reinterpret_cast<float2*>(smem + lay.tw_off);
  float* ie_s = reinterpret_cast<float*>(smem + lay.ie_off);
  uint8_t* codes = smem + lay.codes_off;
  unsigned char* stage = smem + lay.warp_off + warp * lay.warp_bytes;
  float2* ex = reinterpret_cast<float2*>(stage + lay.stage_bytes);
  constexpr int slot_bytes = kTwSlotB;

  for (int i = tid; i < N; i += NT) {
    const float2 w = __ldg(p.twP + i);
    tws[i] = w;
  }
  if (tid == 0) *abort_flag = 0;
  if (lane == 0) {
    for (int s = 0; s < K; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_base), kWTmemCols);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  // this warp's columns: 256 columns of its lane quarter
  const uint32_t tE = *tmem_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                      static_cast<uint32_t>((warp >> 2) * kTwTmemWarp);
  uint64_t pol = 0;
  if (lane == 0) pol = evict_first_policy();
  pol = __shfl_sync(0xffffffffu, pol, 0);
  float zero[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) zero[i] = 0.f;

  const int nch = warp < p.chunks ? (p.chunks - 1 - warp) / NW + 1 : 0;
  // start the warps of the upper half a little later, so that the two warps
  // sharing a scheduler tend to be in different phases of their steps
  if (warp >= 4) __nanosleep(1400);
  int issued = 0;  // steps whose copies this warp has issued
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
    const uint32_t tP = energy_here ? tE + OWN : tE;   // data symbol dl at tP + 2 OWN dl
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
        const int ia = 2 * ipi;
        twin_issue<LOG2N>(p, f, warp + ic * NW, pilot_here, d0, items, ia, stage + is * slot_bytes,
                          smem_u32(&bars[is]), pol, lane);
        // test hook: the first staging phase of block 0 also waits for 16
        // bytes that no copy delivers, so its bounded wait runs out
        if (p.fault == 1 && blockIdx.x == 0 && warp == 0 && g == 0 && s == 0 && lane == 0)
          mbar_expect_tx_only(smem_u32(&bars[is]), 16);
        ++issued;
        is = (is + 1 == K) ? 0 : is + 1;
        if (++ipi == npairs) {
          ipi = 0;
          ++ic;
        }
      }
    }
    for (int lc = 0; lc < nch; ++lc) {
      const int m = (warp + lc * NW) * A + team;   // this lane's antenna
      const bool valid = m < p.M;                  // a chunk's last teams may have none
      const size_t hrow = (static_cast<size_t>(f) * p.Mtot + p.m0 + blockIdx.y * p.shard_y + m) * N;
      float2 h[32];
      if (!pilot_here) {
        // channel written in group 0 (zero for a team without an antenna, so
        // that its stale rows add nothing)
#pragma unroll
        for (int e = 0; e < 32; ++e)
          h[e] = valid ? p.H_out[hrow + bin_of<LOG2N>(jt, e)] : make_float2(0.f, 0.f);
      }
      for (int ip = 0; ip < npairs; ++ip) {
        float2 re[32], im[32];
        wait_slot(smem_u32(&bars[slot]), phase, abort_flag, p.status);
        // both rows; a missing second row leaves earlier samples in the slot
        // (finite integers), whose transform is not used
        const uint32_t* sa =
            reinterpret_cast<const uint32_t*>(stage + slot * slot_bytes) + team * (N + L);
        const uint32_t* sb = sa + kTwHalfB / 4;
        {
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            // sc16 -> float v + 2^23 + 32768 exactly: sign bits flipped to
            // offset binary, each half placed under the exponent bytes of
            // 2^23 (the offset leaves where pass 1 first adds two samples)
            const uint32_t ua = sa[jt + L * r] ^ 0x80008000u;
            const uint32_t ub = sb[jt + L * r] ^ 0x80008000u;
            re[r] = make_float2(__uint_as_float(__byte_perm(ua, 0x4b000000u, 0x7610)),
                                __uint_as_float(__byte_perm(ub, 0x4b000000u, 0x7610)));
            im[r] = make_float2(__uint_as_float(__byte_perm(ua, 0x4b000000u, 0x7632)),
                                __uint_as_float(__byte_perm(ub, 0x4b000000u, 0x7632)));
          }
        }
        unsigned char* const yslot = stage + slot * slot_bytes;
        const uint32_t ybar = smem_u32(&bars[slot]);
        if (++slot == K) {
          slot = 0;
          phase ^= 1;
        }
        // pass 1: 32-point DFTs over n1 (n = jt + L n1)
        twin_dft32_sr<true>(re, im);
        // every lane is done with the exchange of the previous step (and with
        // this step's slot): transpose in one round of 16-byte stores, rows
        // n2 < 16 in the slot just read, the others in the exchange region
        __syncwarp();
        {
          unsigned char* wrow = (lane < 16 ? yslot : reinterpret_cast<unsigned char*>(ex)) + (lane & 15) * kTwXRow;
#pragma unroll
          for (int r = 0; r < 32; ++r)
            *reinterpret_cast<float4*>(wrow + 16 * r) = make_float4(re[r].x, re[r].y, im[r].x, im[r].y);
        }
        __syncwarp();
        // row R = lane holds the pass-1 outputs k1 of team R / L, its thread
        // n2 = R % L; this lane reads k1 = jt + L i, n2 = 0 .. L - 1 of its
        // team into register i L + n2
        if constexpr (L == 32) {
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            const float4 v = *reinterpret_cast<const float4*>(
                (r < 16 ? yslot : reinterpret_cast<const unsigned char*>(ex)) + (r & 15) * kTwXRow + 16 * lane);
            re[r] = make_float2(v.x, v.y);
            im[r] = make_float2(v.z, v.w);
          }
        } else {
          // a team's L rows lie in one of the two places (L divides 16)
          const unsigned char* trow = (team * L < 16 ? yslot : reinterpret_cast<const unsigned char*>(ex)) +
                                      ((team * L) & 15) * kTwXRow + 16 * jt;
#pragma unroll
          for (int i = 0; i < 32 / L; ++i) {
#pragma unroll
            for (int n2 = 0; n2 < L; ++n2) {
              const float4 v = *reinterpret_cast<const float4*>(trow + n2 * kTwXRow + 16 * L * i);
              re[i * L + n2] = make_float2(v.x, v.y);
              im[i * L + n2] = make_float2(v.z, v.w);
            }
          }
        }
        __syncwarp();
        if (to_issue > 0 && !*abort_flag) {
          ++issued;
          fence_proxy_async();
          const int ia = 2 * ipi;
          twin_issue<LOG2N>(p, f, warp + ic * NW, pilot_here, d0, items, ia, yslot, ybar, pol, lane);
          --to_issue;
          if (++ipi == npairs) {
            ipi = 0;
            ++ic;
          }
        }
        // pass twiddles W_N^(n2 k1) of register i L + n2, k1 = jt + L i
#pragma unroll
        for (int i = 0; i < 32 / L; ++i) {
#pragma unroll
          for (int n2 = 1; n2 < L; ++n2) {
            const float2 w = tws[n2 * 32 + jt + L * i];
            const int e = i * L + n2;
            const float2 xr = re[e], xi = im[e];
            re[e] = __ffma2_rn(xi, f2(-w.y), __fmul2_rn(xr, f2(w.x)));
            im[e] = __ffma2_rn(xr, f2(w.y), __fmul2_rn(xi, f2(w.x)));
          }
        }
        // pass 2: radix-L DFTs over n2; register e holds bin bin_of(jt, e)
        twin_pass2<L>(re, im);
        const int ia = 2 * ip;
        if (pilot_here && ip == 0) {
          // first row: the pilot.  LS estimate H = Y conj(X) / |X|^2 (1/sqrt(N)
          // folded into xinv); group 0 writes it out and adds |H|^2 into the
          // energy
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int k = bin_of<LOG2N>(jt, e);
            const float2 hv = cmul(make_float2(re[e].x, im[e].x), __ldg(p.xinv + k));
            h[e] = valid ? hv : make_float2(0.f, 0.f);
            if (valid && energy_here) p.H_out[hrow + k] = hv;
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
    // ---- group end: every warp's steps are done, every copy of the group
    // has landed; the per-warp regions are free for the reduction (and the
    // tensor-memory stores of every warp are ordered before the loads of
    // its lane-quarter partner)
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (energy_here) {
      // warps w and w + 4 share a lane quarter: warp w < 4 adds the other's
      // columns in tensor memory, then four warps go through shared memory
      float* RE = reinterpret_cast<float*>(smem + lay.warp_off);   // [4][A][N]
      if (warp < 4) {
        float e[OWN], e2[OWN];
        TmE::ld(tE, e);
        TmE::ld(tE + kTwTmemWarp, e2);
        tmem_wait_ld();
#pragma unroll
        for (int cc = 0; cc < OWN; ++cc) RE[(warp * A + team) * N + bin_of<LOG2N>(jt, cc)] = e[cc] + e2[cc];
      }
      __syncthreads();
      for (int k = tid; k < N; k += NT) {
        float E = 0.f;
#pragma unroll
        for (int w = 0; w < 4 * A; ++w) E += RE[w * N + k];
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
    // the group's data items in tensor memory, block by block (a step's
    // pair of items interleaved in 128 columns, or an item alone in 64):
    // the two warps of a lane quarter take alternate blocks, add both
    // warps' sums and write them to shared memory: [4][A][nd][N]
    static_assert(kTwDg0 <= kTwDg, "a group's data items fit one reduction");
    float2* RP = reinterpret_cast<float2*>(smem + lay.warp_off);
    const int dlc = kTwDg;
    const int dl0 = 0;
    const int n = nd;
    {
      const uint32_t tfirst = tE - static_cast<uint32_t>((warp >> 2) * kTwTmemWarp);   // first warp's columns
      const int j0 = pilot_here ? 1 : 0;
      int blk = 0;
      for (int it = j0; it < items; ++blk) {
        bool pr;
        const uint32_t tb = tfirst + (tP - tE) + twin_block_col(it, pilot_here, &pr, items);
        if ((blk & 1) == (warp >> 2)) {
          float2* dst = RP + static_cast<size_t>(((warp & 3) * A + team) * dlc + (it - j0)) * N;
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
                dst[bin_of<LOG2N>(jt, q0 / 2 + i)] = make_float2(t[2 * i] + t2[2 * i], t[2 * i + 1] + t2[2 * i + 1]);
            }
          }
        }
        it += pr ? 2 : 1;
      }
    }
    {
      __syncthreads();
      // four items per thread at a time: their shared-memory sums are all
      // loaded before the first is demapped; one copy of the loop per
      // constellation, so that the slicer inside it has no branches
      auto demap_items = [&](auto tcount) {
        constexpr int T = decltype(tcount)::value;
        for (int idx0 = tid; idx0 < n * N; idx0 += 4 * NT) {
          float2 sv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int idx = min(idx0 + u * NT, n * N - 1);
            const int j = idx >> LOG2N;
            const int k = idx & (N - 1);
            sv[u] = make_float2(0.f, 0.f);
#pragma unroll
            for (int w = 0; w < 4 * A; ++w) sv[u] = cadd(sv[u], RP[static_cast<size_t>(w * dlc + j) * N + k]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int idx = idx0 + u * NT;
            if (idx >= n * N) break;
            const int j = idx >> LOG2N;
            const int k = idx & (N - 1);
            const float2 s = sv[u];
            const int dl = dl0 + j;
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
      for (int it = tid; it < items8; it += NT) {
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
  if (lane == 0 && *abort_flag) {
    // a wait gave up: give any copy of this warp still in flight a bounded
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
