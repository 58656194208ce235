// lsas_warp.cuh -- per-warp fused receiver kernel for N <= 1024.
//
// One block per frame, NW warps, each an independent pipeline over whole
// antenna-symbol rows.  Warp w takes antenna chunks w, w + NW, ... (A =
// 32/L antennas per chunk; L = N/32 lanes form one antenna's FFT team).  Per
// step a warp
//   * waits for its staging slot (bulk asynchronous copy of the CP-stripped
//     rows, the CP removal of Sec. II-B done as addressing) and refills it
//     K steps ahead,
//   * runs the radix-32 pass in registers, transposes through its own
//     padded exchange region (only __syncwarp), applies the pass twiddles
//     and runs the radix-L pass,
//   * pilot: LS estimate H = Y conj(X) / |X|^2 (Sec. II-C), written out and
//     kept in registers, and |H|^2 added to the channel energy;
//     data symbol: conj(H) Y (Sec. II-C), summed over the chunk's antennas
//     with shuffles,
//   * accumulates per subcarrier in the warp's own tensor-memory columns.
// Warps never wait for each other inside a data-symbol group.  At a group's
// end the block adds the warps' partial sums in warp order through shared
// memory (the staging rings are idle then), forms z = P / E and demaps
// (Sec. II-B), or writes the block's partial sums (antenna split).
#pragma once

#include "lsas_kernels.cuh"

namespace lsas {

#ifdef __CUDACC__

// Issue the bulk copies of one warp step (antennas of chunk c, symbol s)
// into a slot: lane 0 registers the byte count, lane a copies row a.
template <int LOG2N, bool FC32>
__device__ __forceinline__ void wissue(const KParams& p, int f, int c, int s,
                                       unsigned char* slot, int team_stage, uint32_t bar,
                                       uint64_t pol, int lane) {
  constexpr int N = 1 << LOG2N, A = wgeo_A(N);
  constexpr uint32_t bytes = N * (FC32 ? 8 : 4);
  const int nvalid = min(A, p.M - c * A);
  if (lane == 0) mbar_expect_tx(bar, bytes * nvalid);
  for (int a = lane; a < nvalid; a += 32)
    bulk_load(smem_u32(slot + a * team_stage), row_ptr<LOG2N, FC32>(p, f, c * A + a, s), bytes,
              bar, pol);
}

// Symbol index of item `it` of a chunk in a data-symbol group starting at
// data symbol d0 (the pilot first when the group transforms it).
__device__ __forceinline__ int witem_symbol(const KParams& p, bool pilot_here, int d0, int it) {
  if (pilot_here) {
    if (it == 0) return p.pilot_idx;
    --it;
  }
  const int d = d0 + it;
  return d < p.pilot_idx ? d : d + 1;
}

// Load the inputs of the last FFT pass times its twiddles, held in shared
// memory as {w, -j w} pairs (two packed instructions per product).
template <int LOG2N>
__device__ __forceinline__ void wfinal_exchange_read(float2 (&v)[32], const float2* ex, int jt,
                                                     const float4* tw) {
  constexpr int L = (1 << LOG2N) / 32;
#pragma unroll
  for (int i = 0; i < 32 / L; ++i) {
    const int j = jt + i * L;
#pragma unroll
    for (int r = 0; r < L; ++r) {
      const float2 u = ex[xpad(j + 32 * r)];
      if (r == 0) {
        v[i * L + r] = u;
      } else {
        const float4 t = tw[r * 32 + j];
        v[i * L + r] = cmulw(u, make_float2(t.x, t.y), make_float2(t.z, t.w));
      }
    }
  }
}

template <int LOG2N, bool FC32>
__global__ void __launch_bounds__(32 * wgeo_warps(FC32 ? 8 : 4), 1) warp_kernel(const KParams p) {
  constexpr int N = 1 << LOG2N;
  constexpr int NW = wgeo_warps(FC32 ? 8 : 4);   // warps of the block
  constexpr int NT = 32 * NW;
  constexpr int TMW = wgeo_tmem_warp(NW);         // TMEM columns per warp
  constexpr int A = wgeo_A(N), OWN = wgeo_OWN(N), XS = wgeo_XS(N);
  static_assert(N <= 1024, "the per-warp kernel covers N <= 1024");
  using TmP = Tmem<2 * OWN>;   // one data symbol of partial sums (complex)
  using TmE = Tmem<OWN>;       // channel energy
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int alpha = lane % A;   // antenna of the chunk
  const int jt = lane / A;      // FFT team thread
  const int K = p.nslots;
  const WLayout lay = make_wlayout(N, FC32 ? 8 : 4, K, p.dg);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem) + warp * kMaxSlots;
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(smem + kWTmemAddr);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kWAbort);
  float4* tws = reinterpret_cast<float4*>(smem + lay.tw_off);
  float* ie_s = reinterpret_cast<float*>(smem + lay.ie_off);
  uint8_t* codes = smem + lay.codes_off;
  unsigned char* stage = smem + lay.warp_off + warp * lay.warp_bytes;
  float2* ex = reinterpret_cast<float2*>(stage + lay.stage_bytes) + alpha * XS;
  const int slot_bytes = A * lay.team_stage;

  for (int i = tid; i < N; i += NT) {
    const float2 w = __ldg(p.twP + i);
    tws[i] = make_float4(w.x, w.y, -w.y, w.x);
  }
  if (tid == 0) *abort_flag = 0;
  if (lane == 0 && p.use_tma) {
    for (int s = 0; s < K; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_base), kWTmemCols);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  // this warp's columns: TMW columns of its lane quarter
  const uint32_t tE = *tmem_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                      static_cast<uint32_t>((warp >> 2) * TMW);
  const uint32_t tP = tE + OWN;   // data symbol dl at tP + 2 OWN dl
  uint64_t pol = 0;
  if (p.use_tma) {
    if (lane == 0) pol = evict_first_policy();
    pol = __shfl_sync(0xffffffffu, pol, 0);
  }
  // zero-fill of accumulator columns, 16 (or fewer) at a time
  constexpr int ZC = OWN < 16 ? OWN : 16;
  float zero[ZC];
#pragma unroll
  for (int i = 0; i < ZC; ++i) zero[i] = 0.f;

  const int nch = warp < p.chunks ? (p.chunks - 1 - warp) / NW + 1 : 0;
  // start the warps of the upper half a little later, so that the two warps
  // sharing a scheduler tend to be in different phases of their steps
  if (warp >= 4) __nanosleep(1400);
  int step = 0;    // this warp's step counter over the whole frame
  int issued = 0;  // steps whose copies this warp has issued
  int slot = 0;    // ring slot of the next step to consume (step % K) ...
  int phase = 0;   // ... and its mbarrier phase ((step / K) & 1)
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
      for (int q0 = 0; q0 < OWN; q0 += ZC) Tmem<ZC>::st(tE + q0, zero);
    }
    for (int dl = 0; dl < nd; ++dl) {
#pragma unroll
      for (int q0 = 0; q0 < 2 * OWN; q0 += ZC) Tmem<ZC>::st(tP + 2 * OWN * dl + q0, zero);
    }
    // issue cursor: local chunk and item of the next step to stage, and how
    // many steps of this group are still to be staged
    int ic = 0, iit = 0;
    int to_issue = nch * items;
    if (p.use_tma && !*abort_flag) {
      // the ring held generic data (last group's reduction): order it before
      // the copies, then fill the first K slots of this group
      fence_proxy_async();
      int is = slot;
      for (int s = 0; s < K && to_issue > 0; ++s, --to_issue) {
        wissue<LOG2N, FC32>(p, f, warp + ic * NW, witem_symbol(p, pilot_here, d0, iit),
                            stage + is * slot_bytes, lay.team_stage, smem_u32(&bars[is]), pol,
                            lane);
        // test hook: the first staging phase of block 0 also waits for 16
        // bytes that no copy delivers, so its bounded wait runs out
        if (p.fault == 1 && blockIdx.x == 0 && warp == 0 && g == 0 && s == 0 && lane == 0)
          mbar_expect_tx_only(smem_u32(&bars[is]), 16);
        ++issued;
        is = (is + 1 == K) ? 0 : is + 1;
        if (++iit == items) {
          iit = 0;
          ++ic;
        }
      }
    }
    for (int lc = 0; lc < nch; ++lc) {
      const int c = warp + lc * NW;
      const int m = c * A + alpha;
      const bool valid = m < p.M;
      const size_t hrow = (static_cast<size_t>(f) * p.Mtot + p.m0 + blockIdx.y * p.shard_y + m) * N;
      float2 h[32];
      if (!pilot_here) {
        // channel from memory: given (demodulate) or written in group 0
        const float2* Hs = fft_pilot(p) ? p.H_out : p.H_in;
#pragma unroll
        for (int e = 0; e < 32; ++e)
          h[e] = valid ? Hs[hrow + bin_of<LOG2N>(jt, e)] : make_float2(0.f, 0.f);
        if (g == 0) {
          float2 e2[32];
#pragma unroll
          for (int e = 0; e < 32; ++e) e2[e] = make_float2(h[e].x * h[e].x + h[e].y * h[e].y, 0.f);
          reduce_scatter<A, 16>(e2, alpha);
          float acc[OWN];
          tmem_wait_st();
          TmE::ld(tE, acc);
          tmem_wait_ld();
#pragma unroll
          for (int cc = 0; cc < OWN; ++cc) acc[cc] += e2[cc].x;
          TmE::st(tE, acc);
        }
      }
      for (int it = 0; it < items; ++it, ++step) {
        float2 v[32];
        if (p.use_tma) {
          wait_slot(smem_u32(&bars[slot]), phase, abort_flag, p.status);
          if (valid) {
            load_row<LOG2N, FC32>(v, stage + slot * slot_bytes + alpha * lay.team_stage, jt, false);
          } else {
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
          }
        } else {
          if (valid) {
            load_row<LOG2N, FC32>(v, row_ptr<LOG2N, FC32>(p, f, m, witem_symbol(p, pilot_here, d0, it)),
                                  jt, true);
          } else {
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
          }
        }
        // every lane is done with the slot (and with the exchange of the
        // previous step): refill the slot K steps ahead
        __syncwarp();
        if (p.use_tma && to_issue > 0 && !*abort_flag) {
          ++issued;
          fence_proxy_async();
          wissue<LOG2N, FC32>(p, f, warp + ic * NW, witem_symbol(p, pilot_here, d0, iit),
                              stage + slot * slot_bytes, lay.team_stage, smem_u32(&bars[slot]),
                              pol, lane);
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
        dft<32, true>(v, p);
        final_exchange_write<LOG2N>(v, ex, jt);
        __syncwarp();
        wfinal_exchange_read<LOG2N>(v, ex, jt, tws);
        final_dft<LOG2N, true>(v, p);
        if (pilot_here && it == 0) {
          // LS estimate H = Y conj(X) / |X|^2 (1/sqrt(N) folded into xinv)
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int k = bin_of<LOG2N>(jt, e);
            const float2 hv = cmul(v[e], __ldg(p.xinv + k));
            h[e] = valid ? hv : make_float2(0.f, 0.f);
            if (valid && g == 0) p.H_out[hrow + k] = hv;
            v[e] = make_float2(h[e].x * h[e].x + h[e].y * h[e].y, 0.f);
          }
          reduce_scatter<A, 16>(v, alpha);
          float acc[OWN];
          tmem_wait_st();
          TmE::ld(tE, acc);
          tmem_wait_ld();
#pragma unroll
          for (int cc = 0; cc < OWN; ++cc) acc[cc] += v[cc].x;
          TmE::st(tE, acc);
        } else {
          // MRC numerator: conj(H) Y summed over the chunk's antennas
          const int dl = it - (pilot_here ? 1 : 0);
          const uint32_t tp = tP + 2 * OWN * dl;
          if constexpr (A == 1) {
            // one antenna per step: fuse the product into the accumulation,
            // P += conj(H) Y as four FMAs per subcarrier
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
          } else {
            // several antennas per step: sum them with shuffles first
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = cmulc(h[e], v[e]);
            reduce_scatter<A, 16>(v, alpha);
            tmem_wait_st();
#pragma unroll
            for (int q0 = 0; q0 < 2 * OWN; q0 += (2 * OWN < 16 ? 2 * OWN : 16)) {
              constexpr int QC = 2 * OWN < 16 ? 2 * OWN : 16;
              float acc[QC];
              Tmem<QC>::ld(tp + q0, acc);
              tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < QC / 2; ++i) {
                acc[2 * i] += v[q0 / 2 + i].x;
                acc[2 * i + 1] += v[q0 / 2 + i].y;
              }
              Tmem<QC>::st(tp + q0, acc);
            }
          }
        }
      }
    }
    tmem_wait_st();
    // ---- group end: every warp's steps are done, every copy of the group
    // has landed; the per-warp regions are free for the reduction
    __syncthreads();
    if (g == 0) {
      float* RE = reinterpret_cast<float*>(smem + lay.warp_off);   // [NW][N]
      float e[OWN];
      TmE::ld(tE, e);
      tmem_wait_ld();
#pragma unroll
      for (int cc = 0; cc < OWN; ++cc) RE[warp * N + bin_of<LOG2N>(jt, alpha * OWN + cc)] = e[cc];
      __syncthreads();
      for (int k = tid; k < N; k += NT) {
        float E = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) E += RE[w * N + k];
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
    float2* RP = reinterpret_cast<float2*>(smem + lay.warp_off);   // [NW][dlc][N]
    const int dlc = min(nd, lay.warp_bytes / (N * 8));
    for (int dl0 = 0; dl0 < nd; dl0 += dlc) {
      const int n = min(dlc, nd - dl0);
      for (int j = 0; j < n; ++j) {
        float acc[2 * OWN];
        TmP::ld(tP + 2 * OWN * (dl0 + j), acc);
        tmem_wait_ld();
        float2* dst = RP + static_cast<size_t>(warp * dlc + j) * N;
#pragma unroll
        for (int cc = 0; cc < OWN; ++cc)
          dst[bin_of<LOG2N>(jt, alpha * OWN + cc)] = make_float2(acc[2 * cc], acc[2 * cc + 1]);
      }
      __syncthreads();
      for (int idx = tid; idx < n * N; idx += NT) {
        const int j = idx >> LOG2N;
        const int k = idx & (N - 1);
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < NW; ++w) s = cadd(s, RP[static_cast<size_t>(w * dlc + j) * N + k]);
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
  if (lane == 0 && p.use_tma && *abort_flag) {
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
