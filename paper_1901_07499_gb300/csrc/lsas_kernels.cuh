// lsas_kernels.cuh -- device code of liblsas for sm_103a.
//
// One FFT team of L = N/32 threads transforms one N-point OFDM symbol of one
// antenna, 32 complex points per thread in registers: a Stockham auto-sort
// FFT, radix 32 then radix N/32 (N = 2048: 32 x 8 x 8), exchanging data
// between passes through padded shared memory.  A warp's lanes hold A
// antennas x F = 32/A sub-lanes, so a warp group of W warps holds the teams
// of A antennas (A = 128/L, at most 32), and the sum over antennas of MRC is
// a warp-shuffle reduction.
//
// Input samples are staged by bulk asynchronous copies (cp.async.bulk, the
// TMA engine) into a ring of shared-memory slots, one contiguous CP-stripped
// symbol row per antenna, completion tracked by mbarriers: the CP removal of
// Sec. II-B done as addressing.  Every wait on an mbarrier is bounded: after
// ~2 s it latches LSAS_ERR_TIMEOUT and the block runs on without waiting
// again, so a missing completion can never hang the GPU.
//
//   frame_kernel    one block per frame, warp-specialised: a producer warp
//                   group stages rows, converts them and runs the first FFT
//                   pass(es); a consumer warp group runs the last pass, forms
//                   the LS estimate from the pilot (Sec. II-C), multiplies
//                   every data symbol by conj(H), sums over antennas with
//                   shuffles and accumulates per subcarrier in tensor memory
//                   (the conjugate and the channel-energy sum are formed once
//                   per frame and reused, Sec. III), then z = sum / energy ->
//                   Gray slicer -> packed bits.  The two groups hand the
//                   pass boundary over through a double-buffered exchange.
//   estimate_kernel one warp group per (frame, antenna chunk): pilot -> H.
//   fft_kernel      one warp group per (frame, antenna chunk): symbols -> Y.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lsas {

// kModePartial: the fused path of one antenna shard, stopping at the MRC
// partial sums (the antenna split of the distributed receiver, Sec. IV).
enum { kModeEstimate = 0, kModeDemod = 1, kModeRun = 2, kModePartial = 3 };
enum { kStOk = 0, kStTimeout = 6, kStDevice = 7 };

constexpr int kMaxSlots = 6;
constexpr int kSmemHeader = 256;     // mbarriers, TMEM address, flags
constexpr int kMaxThresholds = 15;   // 256-QAM: 16 levels per axis

struct KParams {
  const void* in;        // [F][M][S][N+CP] samples (sc16 or fc32)
  float2* H_out;         // [F][M][N]
  const float2* H_in;    // [F][M][N] (demodulate)
  uint8_t* bits;         // [F][D*N*q/8]
  float2* eq;            // [F][D][N] or null
  float2* Y_out;         // [F][M][S][N] (fft)
  const float2* twP;     // pass twiddles W (layout: pass_tw_count)
  const float2* xinv;    // conj(X[k]) / |X[k]|^2 / sqrt(N)
  int* status;           // latched device status
  float2* P_out;         // [F][D][N] shard partial sum conj(H) Y (partial)
  float* E_out;          // [F][N]    shard partial sum |H|^2 (partial)
  const float2* P_in;    // [G][F][D][N] partials to combine
  const float* E_in;     // [G][F][N]
  int M;                 // antennas this call processes
  int m0, Mtot;          // first of them, antennas per frame in the arrays
  int N, S, cp, pilot_idx, D;
  int shards, nframes;   // combine: partials per frame, frames; tensor-core FFT: rows
  const void* tc_w1;     // tensor-core FFT: 32-point DFT operand images (hi, lo)
  const void* tc_w2;     //   N/32-point DFT operand images (hi, lo)
  const float2* tc_tw;   //   inter-stage twiddles W_N^(n2 k1), [n2][k1]
  int terms;             //   1: plain operands; 3: hi+lo split operands
  int tc_bf16;           //   0: fp16 operands; 1: bf16
  const float* pn;       // packet detection: PN chips (real), pn_len of them
  int pn_len, cap_len, window, backoff;
  int* offsets;          //   per frame: detected preamble start (out)
  float* peaks;          //   per frame: correlation power at it (out, nullable)
  const int* offsets_in; //   per frame: preamble start (extraction)
  int fault;             // test hook: 1 = block 0 waits for 16 bytes that never come
  int hybrid;            // N = 1024, sc16, staged: second FFT pass on the tensor cores
  int twin;              // N = 1024, sc16, staged: two symbols per step (twin_kernel)
  int shard_y;           // partial mode, one launch for all shards: antennas per grid row
                         // blockIdx.y (its first antenna is m0 + blockIdx.y * shard_y, its
                         // partials start at shard blockIdx.y of [G][F][...]); 0 otherwise
  int grid_y;            // grid rows (shards) of the launch; 0 or 1 for a 1-D grid
  int group_z;           // partial mode of the per-warp kernel: 1 = grid z index g runs
                         // data-symbol group g alone (groups grid layers); 0 otherwise
  int chunks;            // ceil(M / A)
  int groups, dg;        // data-symbol groups per frame, data symbols per group
  int mode;              // kModeDemod, kModeRun or kModePartial (frame_kernel)
  int use_tma, nslots;
  int tmem_cols, tmem_cth;   // TMEM allocation (columns) and columns per thread
  int q, wbits, axes, nthr;
  float inv_sqrtN;
  float thr[kMaxThresholds];   // per-axis decision boundaries (float32)
  float2 w32[16];              // W_32^e = {cos, -sin}(2 pi e / 32), e < 16
  float2 w32n[16];             // {-Im, Re} of W_32^e (packed complex multiply)
};

// ---------------------------------------------------------------- geometry

__host__ __device__ constexpr int geo_L(int N) { return N / 32; }
__host__ __device__ constexpr int geo_A(int N) { return 128 / (N / 32) > 32 ? 32 : 128 / (N / 32); }
__host__ __device__ constexpr int geo_F(int N) { return 32 / geo_A(N); }
__host__ __device__ constexpr int geo_W(int N) { return geo_L(N) / geo_F(N); }
__host__ __device__ constexpr int geo_TW(int N) { return 32 * geo_W(N); }
__host__ __device__ constexpr int geo_T(int N) { return 2 * geo_TW(N); }
__host__ __device__ constexpr int geo_OWN(int N) { return 32 / geo_A(N); }
// exchange stride (float2): N plus one pad per 32, rounded so that antenna
// regions start 16/A float2 apart modulo the 16 bank pairs (A <= 16)
__host__ __device__ constexpr int geo_XS(int N) {
  return geo_A(N) > 16 ? (N + N / 32)
                       : (N + N / 32) + ((16 / geo_A(N) - (N + N / 32) % 16) + 16) % 16;
}
// staging stride pad (samples) per antenna: rows start F (sc16) or F/2
// (fc32) words of banks apart, and stay 16-byte aligned for bulk copies
__host__ __device__ constexpr int geo_spad(int N, int bps) {
  return bps == 4 ? (geo_F(N) < 4 ? 4 : geo_F(N)) : (geo_F(N) / 2 < 2 ? 2 : geo_F(N) / 2);
}

template <int LOG2N>
struct Geo {
  static constexpr int N = 1 << LOG2N;
  static constexpr int L = geo_L(N);      // threads per FFT team
  static constexpr int A = geo_A(N);      // antennas per step
  static constexpr int F = geo_F(N);      // sub-lanes per warp
  static constexpr int W = geo_W(N);      // warps per warp group
  static constexpr int TW = geo_TW(N);    // threads per warp group
  static constexpr int T = geo_T(N);      // threads of the fused kernel
  static constexpr int OWN = geo_OWN(N);  // subcarriers per thread after the reduction
  static constexpr int XS = geo_XS(N);
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Shared memory: header, pass twiddles of the last pass (N <= 1024), the
// staging ring, the final-pass exchange (two buffers in the fused kernel) and,
// for N = 2048, the producer's middle-pass exchange.  After the chunk loop of
// the fused kernel the staging ring holds the demapped codes.
struct Layout {
  int tw_off;
  int stage_off;
  int team_stage;   // bytes per antenna per slot
  int ex_off;       // final-pass exchange buffer(s), A * XS float2 each
  int ex1_off;      // N = 2048: middle-pass exchange
  int codes_off;    // fused kernel, after the loop: uint8[dg][N]
  int total;
};

__host__ __device__ inline Layout make_layout(int N, int bps, int nslots, int nex) {
  Layout l;
  const int A = geo_A(N);
  l.tw_off = kSmemHeader;
  l.stage_off = align_up(l.tw_off + (N <= 1024 ? N * 8 : 0), 128);
  l.team_stage = (N + geo_spad(N, bps)) * bps;
  l.ex_off = align_up(l.stage_off + nslots * A * l.team_stage, 128);
  l.ex1_off = l.ex_off + nex * A * geo_XS(N) * 8;
  l.total = align_up(l.ex1_off + (N > 1024 ? A * geo_XS(N) * 8 : 0), 128);
  l.codes_off = l.stage_off;
  return l;
}

// Tensor memory of the fused kernel: the consumer warps (one per TMEM lane
// quarter) keep OWN subcarriers of partial sums for dg data symbols
// (complex) plus the channel energy, per thread.
__host__ __device__ inline int tmem_cols_thread(int N, int dg) {
  return 2 * geo_OWN(N) * dg + geo_OWN(N);
}
__host__ __device__ inline int tmem_alloc_cols(int N, int dg) {
  int c = 32;
  while (c < tmem_cols_thread(N, dg)) c *= 2;
  return c;
}

// Number of pass twiddles in the host-built table (layout in pass_twiddles):
// N <= 1024: [r][j] = W_N^(j r), r < N/32, j < 32 (second pass);
// N = 2048:  [r][j] = W_2048^(8 j r), j < 32 (second pass), then
//            [256 + r*256 + j] = W_2048^(j r), j < 256 (third pass).
__host__ __device__ inline int pass_tw_count(int N) { return N <= 1024 ? N : 256 + 2048; }

// ------------------------------------------------ warp kernel geometry
//
// The per-warp fused kernel (N <= 1024, lsas_warp.cuh): each of its warps
// transforms A = 32/L antenna rows per step on its own (the FFT team of one
// antenna is L = N/32 lanes of one warp), with its own staging ring and
// exchange region; the block synchronises only at data-symbol group ends.
// 8 warps (2 per scheduler): 12 would need <= 168 registers (the N = 1024
// kernel then spills) and leave room for only a 2-slot staging ring, and
// measured slower.
__host__ __device__ constexpr int wgeo_warps(int /*bps*/) { return 8; }
constexpr int kWMaxWarps = 12;
constexpr int kWTmemAddr = kWMaxWarps * kMaxSlots * 8;   // after the mbarriers
constexpr int kWAbort = kWTmemAddr + 16;
constexpr int kWHeader = 640;      // mbarriers [warps][kMaxSlots], TMEM address, flags
constexpr int kWTmemCols = 512;    // all of TMEM, split between the warps
// TMEM columns per warp: warps w, w+4, ... share lane quarter w % 4
__host__ __device__ constexpr int wgeo_tmem_warp(int warps) { return warps > 8 ? 160 : 256; }

__host__ __device__ constexpr int wgeo_A(int N) { return 32 / (N / 32); }
__host__ __device__ constexpr int wgeo_OWN(int N) { return N / 32; }
// exchange stride (float2) per antenna: N plus one pad per 32, rounded so
// that the antenna regions of a warp start 16/A float2 apart modulo 16
__host__ __device__ constexpr int wgeo_XS(int N) {
  return (N + N / 32) +
         (((16 / wgeo_A(N)) % 16 - (N + N / 32) % 16) + 16) % 16;
}
// staging pad (samples) per antenna row: rows start L words of banks apart
// (sc16) or L/2 bank pairs (fc32) and stay 16-byte aligned
__host__ __device__ constexpr int wgeo_spad(int N, int bps) {
  return bps == 4 ? (N / 32 >= 4 ? N / 32 : 4) : (N / 32 >= 4 ? N / 64 : 2);
}

// Shared memory of the warp kernel: header, last-pass twiddles (each as the
// pair {w, -j w} for the packed multiply), 1/E per subcarrier, the demapped
// codes of one group, then one region per warp (staging ring + exchange).
// At group ends the per-warp regions together hold the warps' partial sums
// for the cross-warp reduction.
struct WLayout {
  int tw_off, ie_off, codes_off, warp_off;
  int team_stage;    // bytes per antenna row in a slot
  int stage_bytes;   // one warp's ring
  int warp_bytes;    // one warp's region
  int total;
};
__host__ __device__ inline WLayout make_wlayout(int N, int bps, int nslots, int dg) {
  const int warps = wgeo_warps(bps);
  WLayout l;
  l.tw_off = kWHeader;
  l.ie_off = l.tw_off + N * 16;
  l.codes_off = l.ie_off + N * 4;
  l.warp_off = align_up(l.codes_off + dg * N, 128);
  l.team_stage = (N + wgeo_spad(N, bps)) * bps;
  l.stage_bytes = nslots * wgeo_A(N) * l.team_stage;
  l.warp_bytes = align_up(l.stage_bytes + wgeo_A(N) * wgeo_XS(N) * 8, 128);
  l.total = l.warp_off + warps * l.warp_bytes;
  return l;
}
// data symbols per group that the per-warp TMEM columns hold
__host__ __device__ inline int wgeo_dg_max(int N, int bps) {
  return (wgeo_tmem_warp(wgeo_warps(bps)) - wgeo_OWN(N)) / (2 * wgeo_OWN(N));
}

#ifdef __CUDACC__

// ------------------------------------------------------- PTX primitives

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
// Raise the byte count a phase waits for, without arriving.
__device__ __forceinline__ void mbar_expect_tx_only(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src,
                                          uint32_t bytes, uint32_t bar,
                                          uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: false after ~2 s without completion.
static __device__ __noinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > 2000000000ull) return false;
  }
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ------------------------------------------------------- tensor memory

__device__ __forceinline__ void tmem_alloc(uint32_t smem_dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_dst),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Load / store NC consecutive 32-bit columns of this thread's TMEM lane
// (32x32b shape: thread i of the warp accesses lane base + i).
template <int NC> struct Tmem;
template <> struct Tmem<1> {
  static __device__ __forceinline__ void ld(uint32_t t, float* v) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(t) : "memory");
    v[0] = __uint_as_float(r);
  }
  static __device__ __forceinline__ void st(uint32_t t, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(t),
                 "r"(__float_as_uint(v[0])) : "memory");
  }
};
template <> struct Tmem<2> {
  static __device__ __forceinline__ void ld(uint32_t t, float* v) {
    uint32_t r[2];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(t) : "memory");
    for (int i = 0; i < 2; ++i) v[i] = __uint_as_float(r[i]);
  }
  static __device__ __forceinline__ void st(uint32_t t, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(t),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])) : "memory");
  }
};
template <> struct Tmem<4> {
  static __device__ __forceinline__ void ld(uint32_t t, float* v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(t) : "memory");
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
  }
  static __device__ __forceinline__ void st(uint32_t t, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(t),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])) : "memory");
  }
};
template <> struct Tmem<8> {
  static __device__ __forceinline__ void ld(uint32_t t, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]) : "r"(t) : "memory");
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
  }
  static __device__ __forceinline__ void st(uint32_t t, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(t),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])) : "memory");
  }
};
template <> struct Tmem<16> {
  static __device__ __forceinline__ void ld(uint32_t t, float* v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]) : "r"(t) : "memory");
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
  }
  static __device__ __forceinline__ void st(uint32_t t, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 "
                 "[%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(t),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                 "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                 "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                 "r"(__float_as_uint(v[15])) : "memory");
  }
};

// 32 columns as two 16-column halves
template <> struct Tmem<32> {
  static __device__ __forceinline__ void ld(uint32_t t, float* v) {
    Tmem<16>::ld(t, v);
    Tmem<16>::ld(t + 16, v + 16);
  }
  static __device__ __forceinline__ void st(uint32_t t, const float* v) {
    Tmem<16>::st(t, v);
    Tmem<16>::st(t + 16, v + 16);
  }
};

// ------------------------------------------------------- tcgen05 MMA

// Shared-memory operand descriptor, no swizzle: start address, byte offset
// between core matrices adjacent along K (lbo) and between 8-row groups (sbo).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = static_cast<uint64_t>((addr & 0x3FFFF) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32;
  d |= static_cast<uint64_t>(1) << 46;   // descriptor version
  return d;
}
// kind::f16 instruction descriptor: fp32 accumulator, A and B both fp16 or
// both bf16, K-major, M = 128, n columns.
__device__ __forceinline__ uint32_t umma_idesc(int n, bool bf16) {
  const uint32_t ab = bf16 ? 1u : 0u;
  return (1u << 4) | (ab << 7) | (ab << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(128 >> 4) << 24);
}
__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
               :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(bar) : "memory");
}

// 64 columns as two 32-column halves
template <> struct Tmem<64> {
  static __device__ __forceinline__ void ld(uint32_t t, float* v) {
    Tmem<32>::ld(t, v);
    Tmem<32>::ld(t + 32, v + 32);
  }
  static __device__ __forceinline__ void st(uint32_t t, const float* v) {
    Tmem<32>::st(t, v);
    Tmem<32>::st(t + 32, v + 32);
  }
};

// ------------------------------------------------------- complex helpers

// Complex arithmetic on {re, im} pairs with the packed f32x2 instructions:
// one issue slot per complex add, two per complex multiply.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// a * w with w = {Re, Im} and wn = {-Im, Re}
__device__ __forceinline__ float2 cmulw(float2 a, float2 w, float2 wn) {
  return __ffma2_rn(make_float2(a.x, a.x), w, __fmul2_rn(make_float2(a.y, a.y), wn));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(h) * y
__device__ __forceinline__ float2 cmulc(float2 h, float2 y) {
  return make_float2(h.x * y.x + h.y * y.y, h.x * y.y - h.y * y.x);
}

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }
__host__ __device__ constexpr int brev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

// b * W_32^e for a compile-time e in [0, 16): free for e = 0 and -j, two
// packed instructions otherwise.  W8SUM: the eighth roots W_8 and W_8^3 as
// a sum and a difference scaled by 1/sqrt(2) instead (three instructions
// but a shorter chain; which is faster depends on the kernel, so each
// kernel picks the form that measured faster).
template <bool W8SUM>
__device__ __forceinline__ float2 tw32(float2 b, int e, const KParams& p) {
  constexpr float kS = 0.70710678118654752440f;  // 1/sqrt(2)
  if (e == 0) return b;
  if (e == 8) return make_float2(b.y, -b.x);                                     // -j
  if (W8SUM && e == 4) return __fmul2_rn(make_float2(b.x + b.y, b.y - b.x), make_float2(kS, kS));
  if (W8SUM && e == 12) return __fmul2_rn(make_float2(b.y - b.x, -(b.x + b.y)), make_float2(kS, kS));
  return cmulw(b, p.w32[e], p.w32n[e]);
}

// One radix-2 decimation-in-time stage of half-span S on R registers.
template <int R, int S, bool W8SUM>
__device__ __forceinline__ void dit_stage(float2* a, const KParams& p) {
#pragma unroll
  for (int base = 0; base < R; base += 2 * S) {
#pragma unroll
    for (int i = 0; i < S; ++i) {
      const float2 b = tw32<W8SUM>(a[base + i + S], i * (16 / S), p);
      const float2 x = a[base + i];
      a[base + i] = cadd(x, b);
      a[base + i + S] = csub(x, b);
    }
  }
}
template <int R, int S, bool W8SUM>
__device__ __forceinline__ void dit_stages(float2* a, const KParams& p) {
  if constexpr (S < R) {
    dit_stage<R, S, W8SUM>(a, p);
    dit_stages<R, 2 * S, W8SUM>(a, p);
  }
}

// In-register R-point DFT (R <= 32), natural order in and out: radix-2
// decimation in time over bit-reversed register indices (free renaming).
template <int R, bool W8SUM = false>
__device__ __forceinline__ void dft(float2* v, const KParams& p) {
  constexpr int LOGR = ilog2c(R);
  float2 a[R];
#pragma unroll
  for (int i = 0; i < R; ++i) a[i] = v[brev(i, LOGR)];
  dit_stages<R, 1, W8SUM>(a, p);
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = a[i];
}


// Padded exchange index: one float2 of padding after every 32 entries, so
// that both the row writes (t*32 + r) and the column reads (j + 32 r) of a
// transpose hit distinct banks, and every address is a per-thread base plus
// a compile-time offset.
__device__ __forceinline__ int xpad(int n) { return n + (n >> 5); }

__device__ __forceinline__ void bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Bin k held in register e after the last FFT pass, for team thread t.
template <int LOG2N>
__device__ __forceinline__ int bin_of(int t, int e) {
  using G = Geo<LOG2N>;
  if constexpr (G::N <= 1024) {
    return t + (e / G::L) * G::L + 32 * (e % G::L);
  } else {
    return t + 64 * (e / 8) + 256 * (e % 8);
  }
}

// One interleaved int16 IQ word -> {I, Q} as floats, exactly, without the
// conversion unit: flipping the sign bits gives offset-binary u = v + 32768,
// a byte permute places each half under the exponent bytes of 2^23 (the
// float 2^23 + u), and one packed subtraction of 2^23 + 32768 leaves v.
__device__ __forceinline__ float2 sc16_to_float2(uint32_t w) {
  const uint32_t u = w ^ 0x80008000u;
  const uint32_t lo = __byte_perm(u, 0x4b000000u, 0x7610);
  const uint32_t hi = __byte_perm(u, 0x4b000000u, 0x7632);
  return __fadd2_rn(make_float2(__uint_as_float(lo), __uint_as_float(hi)),
                    make_float2(-8421376.0f, -8421376.0f));
}

// Pass-1 inputs x[jt + r L], r < 32, of one antenna-symbol row (N samples).
template <int LOG2N, bool FC32>
__device__ __forceinline__ void load_row(float2 (&v)[32], const void* row, int jt,
                                         bool from_global) {
  using G = Geo<LOG2N>;
  if constexpr (FC32) {
    const float2* s = static_cast<const float2*>(row);
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = from_global ? __ldg(s + jt + r * G::L) : s[jt + r * G::L];
  } else {
    const uint32_t* s = static_cast<const uint32_t*>(row);
#pragma unroll
    for (int r = 0; r < 32; ++r)
      v[r] = sc16_to_float2(from_global ? __ldg(s + jt + r * G::L) : s[jt + r * G::L]);
  }
}

// N = 2048 only: the middle radix-8 pass, producer side.  v holds pass-1
// outputs (Y1[jt*32 + r]); ex1 is this antenna's middle exchange; sync()
// synchronises the team.  On return v holds the pass-2 outputs of the
// butterflies j = jt + 64 i, i < 4.
template <int LOG2N, typename Sync>
__device__ __forceinline__ void middle_pass(float2 (&v)[32], float2* ex1, int jt,
                                            const float2* tw, const KParams& p, Sync&& sync) {
  if constexpr (Geo<LOG2N>::N > 1024) {
#pragma unroll
    for (int r = 0; r < 32; ++r) ex1[xpad(jt * 32 + r)] = v[r];
    sync();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = jt + 64 * i;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float2 u = ex1[xpad(j + 256 * r)];
        v[i * 8 + r] = (r == 0) ? u : cmul(u, __ldg(tw + r * 32 + (j & 31)));
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) dft<8>(v + i * 8, p);
  }
}

// Twiddles the producer applies before the last exchange (N <= 1024): the
// factor W_N^(j r) of element Y1[j + 32 r] belongs to writer jt = r, output
// k1 = j, i.e. W_N^(jt k1) for its register k1.  They depend only on jt.
template <int LOG2N>
__device__ __forceinline__ void writer_twiddles(float2 (&w)[32], int jt, const float2* tw) {
  using G = Geo<LOG2N>;
  static_assert(G::N <= 1024, "writer-side twiddles are for the two-pass FFT");
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1)
    w[k1] = (jt == 0 || k1 == 0) ? make_float2(1.f, 0.f) : tw[jt * 32 + k1];
}

// Store the inputs of the last FFT pass into the exchange buffer ex.
template <int LOG2N>
__device__ __forceinline__ void final_exchange_write(const float2 (&v)[32], float2* ex, int jt) {
  if constexpr (Geo<LOG2N>::N <= 1024) {
#pragma unroll
    for (int r = 0; r < 32; ++r) ex[xpad(jt * 32 + r)] = v[r];
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = jt + 64 * i;
#pragma unroll
      for (int r = 0; r < 8; ++r) ex[xpad((j >> 5) * 256 + (j & 31) + 32 * r)] = v[i * 8 + r];
    }
  }
}

// Twiddles of the last FFT pass for team thread jt, in register order (they
// depend only on jt, so a thread loads them once per kernel).
template <int LOG2N>
__device__ __forceinline__ void final_twiddles(float2 (&w)[32], int jt, const float2* tw) {
  using G = Geo<LOG2N>;
  constexpr int L = G::L;
  if constexpr (G::N <= 1024) {
#pragma unroll
    for (int i = 0; i < 32 / L; ++i)
#pragma unroll
      for (int r = 0; r < L; ++r) w[i * L + r] = (r == 0) ? make_float2(1.f, 0.f) : tw[r * 32 + jt + i * L];
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < 8; ++r)
        w[i * 8 + r] = (r == 0) ? make_float2(1.f, 0.f) : __ldg(tw + 256 + r * 256 + jt + 64 * i);
  }
}

// Load the inputs of the last FFT pass, times the register-held twiddles w,
// for team thread jt; the pass itself runs in final_dft.
template <int LOG2N>
__device__ __forceinline__ void final_exchange_read_w(float2 (&v)[32], const float2* ex, int jt,
                                                      const float2 (&w)[32]) {
  using G = Geo<LOG2N>;
  constexpr int L = G::L;
  if constexpr (G::N <= 1024) {
#pragma unroll
    for (int i = 0; i < 32 / L; ++i) {
      const int j = jt + i * L;
#pragma unroll
      for (int r = 0; r < L; ++r) {
        const float2 u = ex[xpad(j + 32 * r)];
        v[i * L + r] = (r == 0) ? u : cmul(u, w[i * L + r]);
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = jt + 64 * i;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float2 u = ex[xpad(j + 256 * r)];
        v[i * 8 + r] = (r == 0) ? u : cmul(u, w[i * 8 + r]);
      }
    }
  }
}

// Load the already-twiddled inputs of the last FFT pass (N <= 1024).
template <int LOG2N>
__device__ __forceinline__ void final_exchange_read_plain(float2 (&v)[32], const float2* ex, int jt) {
  using G = Geo<LOG2N>;
  constexpr int L = G::L;
#pragma unroll
  for (int i = 0; i < 32 / L; ++i)
#pragma unroll
    for (int r = 0; r < L; ++r) v[i * L + r] = ex[xpad(jt + i * L + 32 * r)];
}

// Load the inputs of the last FFT pass (with its twiddles) for team thread
// jt; the pass itself runs in final_dft.
template <int LOG2N>
__device__ __forceinline__ void final_exchange_read(float2 (&v)[32], const float2* ex, int jt,
                                                    const float2* tw) {
  using G = Geo<LOG2N>;
  constexpr int L = G::L;
  if constexpr (G::N <= 1024) {
#pragma unroll
    for (int i = 0; i < 32 / L; ++i) {
      const int j = jt + i * L;
#pragma unroll
      for (int r = 0; r < L; ++r) {
        const float2 u = ex[xpad(j + 32 * r)];
        v[i * L + r] = (r == 0) ? u : cmul(u, tw[r * 32 + j]);
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = jt + 64 * i;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float2 u = ex[xpad(j + 256 * r)];
        v[i * 8 + r] = (r == 0) ? u : cmul(u, __ldg(tw + 256 + r * 256 + j));
      }
    }
  }
}

// Last FFT pass; on return v[e] = Y[bin_of(jt, e)] (unscaled).
template <int LOG2N, bool W8SUM = false>
__device__ __forceinline__ void final_dft(float2 (&v)[32], const KParams& p) {
  using G = Geo<LOG2N>;
  if constexpr (G::N <= 1024) {
#pragma unroll
    for (int i = 0; i < 32 / G::L; ++i) dft<G::L, W8SUM>(v + i * G::L, p);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) dft<8, W8SUM>(v + i * 8, p);
  }
}

// Pass twiddles of the last pass: copied to shared memory when N <= 1024.
template <int LOG2N>
__device__ __forceinline__ const float2* load_pass_twiddles(const KParams& p,
                                                            unsigned char* smem,
                                                            const Layout& lay) {
  using G = Geo<LOG2N>;
  if constexpr (G::N <= 1024) {
    float2* tws = reinterpret_cast<float2*>(smem + lay.tw_off);
    for (int i = threadIdx.x; i < G::N; i += blockDim.x) tws[i] = __ldg(p.twP + i);
    return tws;
  } else {
    return p.twP;
  }
}

// Sum over the A antennas held in lane bits [0, log2 A): a reduce-scatter by
// recursive halving with warp shuffles.  Each round the lane keeps the half
// of its registers selected by one bit of alpha and adds the partner's copy
// of it; on return v[c], c < 32/A, holds the sum for register index
// e = alpha * (32/A) + c.
template <int A, int HALF>
__device__ __forceinline__ void reduce_scatter(float2* v, int alpha) {
  if constexpr (A > 1) {
    constexpr int m = A / 2;
    const bool up = (alpha & m) != 0;
#pragma unroll
    for (int c = 0; c < HALF; ++c) {
      const float2 lo = v[c], hi = v[c + HALF];
      const float2 send = up ? lo : hi;
      const float2 keep = up ? hi : lo;
      float2 recv;
      recv.x = __shfl_xor_sync(0xffffffffu, send.x, m);
      recv.y = __shfl_xor_sync(0xffffffffu, send.y, m);
      v[c] = cadd(keep, recv);
    }
    reduce_scatter<A / 2, HALF / 2>(v, alpha);
  }
}

// ------------------------------------------------------- staging pipeline

// Whether the frame kernel transforms the pilot itself (LS estimate) rather
// than reading a given channel.
__device__ __forceinline__ bool fft_pilot(const KParams& p) {
  return p.mode == kModeRun || p.mode == kModePartial;
}

// Items per antenna chunk in data-symbol group g: the pilot first (group 0 of
// the fused modes), then the group's data symbols.
__device__ __forceinline__ int group_items(const KParams& p, int g) {
  const int nd = min(p.dg, p.D - g * p.dg);
  return nd + ((fft_pilot(p) && g == 0) ? 1 : 0);
}

template <int LOG2N, bool FC32>
__device__ __forceinline__ const unsigned char* row_ptr(const KParams& p, int f, int m,
                                                        int s) {
  constexpr int bps = FC32 ? 8 : 4;
  const size_t row = (static_cast<size_t>(f) * p.Mtot + p.m0 + blockIdx.y * p.shard_y + m) * p.S + s;
  return static_cast<const unsigned char*>(p.in) +
         (row * (Geo<LOG2N>::N + p.cp) + p.cp) * bps;
}

// Issue the bulk copies of one step (antennas of chunk c, symbol s) into a
// slot.  Called by a whole warp: lane 0 registers the byte count on the
// slot's mbarrier and lane a (and a + 32) issues the copy of antenna row a.
template <int LOG2N, bool FC32>
__device__ __forceinline__ void issue_step(const KParams& p, int f, int c, int s,
                                           unsigned char* slot, int team_stage,
                                           uint32_t bar, uint64_t pol, int lane) {
  using G = Geo<LOG2N>;
  constexpr uint32_t bytes = G::N * (FC32 ? 8 : 4);
  const int nvalid = min(G::A, p.M - c * G::A);
  if (lane == 0) mbar_expect_tx(bar, bytes * nvalid);
  for (int a = lane; a < nvalid; a += 32)
    bulk_load(smem_u32(slot + a * team_stage), row_ptr<LOG2N, FC32>(p, f, c * G::A + a, s),
              bytes, bar, pol);
}

// Walks the steps of the fused kernel in order (data-symbol group, antenna
// chunk, item) with O(1) work per step.
struct StepCursor {
  int g, c, it, items;
  __device__ void init(const KParams& p) {
    g = 0;
    c = 0;
    it = 0;
    items = group_items(p, 0);
  }
  __device__ int symbol(const KParams& p) const {
    int i = it;
    if (fft_pilot(p) && g == 0) {
      if (i == 0) return p.pilot_idx;
      --i;
    }
    const int d = g * p.dg + i;
    return d < p.pilot_idx ? d : d + 1;
  }
  __device__ void next(const KParams& p) {
    if (++it < items) return;
    it = 0;
    if (++c < p.chunks) return;
    c = 0;
    ++g;
    items = group_items(p, g < p.groups ? g : 0);
  }
};

__device__ __forceinline__ void latch(int* status, int code) {
  atomicCAS(status, 0, code);
}

// Wait for a slot; on timeout latch the status and stop waiting for good.
__device__ __forceinline__ void wait_slot(uint32_t bar, uint32_t parity,
                                          volatile int* abort_flag, int* status) {
  if (mbar_test_wait(bar, parity)) return;   // usually complete: no suspend
  if (*abort_flag) return;
  if (!mbar_wait_bounded(bar, parity)) {
    *abort_flag = 1;
    latch(status, kStTimeout);
  }
}

// Level of one axis value: boundaries at or below v (ties go up).
// Level of one axis: the number of decision thresholds at or below v (a tie
// goes to the upper level).  The compares are independent and summed
// pairwise for the constellation's threshold count (1, 3, 7 or 15), so the
// slicer is a short tree rather than a chain of dependent additions.
template <int T>
__device__ __forceinline__ int count_ge(float v, const float* thr) {
  if constexpr (T == 1) {
    return v >= thr[0] ? 1 : 0;
  } else {
    constexpr int H = T / 2;
    return count_ge<H>(v, thr) + count_ge<T - H>(v, thr + H);
  }
}
__device__ __forceinline__ int axis_level(float v, const KParams& p) {
  switch (p.nthr) {
    case 1: return count_ge<1>(v, p.thr);
    case 3: return count_ge<3>(v, p.thr);
    case 7: return count_ge<7>(v, p.thr);
    default: return count_ge<kMaxThresholds>(v, p.thr);
  }
}
__device__ __forceinline__ uint32_t gray(int l) { return static_cast<uint32_t>(l ^ (l >> 1)); }

// ======================================================= frame kernel

// Named barriers: 0 = whole block; FULL_b / EMPTY_b hand exchange buffer b
// from producers to consumers and back; PROD synchronises the producers.
enum { kBarFull0 = 1, kBarEmpty0 = 3, kBarProd = 5 };

template <int LOG2N, bool FC32>
__global__ void __launch_bounds__(Geo<LOG2N>::T, 1) frame_kernel(const KParams p) {
  using G = Geo<LOG2N>;
  constexpr int N = G::N, A = G::A, T = G::T, TW = G::TW, F = G::F, W = G::W;
  constexpr int OWN = G::OWN;
  using TmP = Tmem<2 * OWN>;   // one data symbol of partial sums (complex)
  using TmE = Tmem<OWN>;       // channel energy
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const bool producer = warp < W;
  const int ltid = tid % TW;           // thread index within its warp group
  const int lane = tid & 31;
  const int alpha = lane % A;
  const int jt = (ltid >> 5) * F + lane / A;
  const Layout lay = make_layout(N, FC32 ? 8 : 4, p.nslots, 2);
  const float2* tw = load_pass_twiddles<LOG2N>(p, smem, lay);
  const int K = p.nslots;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(smem + 160);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 192);
  unsigned char* stage = smem + lay.stage_off;
  float2* ex0 = reinterpret_cast<float2*>(smem + lay.ex_off) + alpha * G::XS;
  float2* ex1 = reinterpret_cast<float2*>(smem + lay.ex1_off) + alpha * G::XS;
  const int slot_bytes = A * lay.team_stage;

  if (tid == 0) {
    *abort_flag = 0;
    if (p.use_tma) {
      for (int s = 0; s < K; ++s) mbar_init(smem_u32(&bars[s]), 1);
      fence_mbar_init();
    }
  }
  if (warp == W) tmem_alloc(smem_u32(tmem_base), p.tmem_cols);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();

  int step = 0;     // global step counter (both groups walk the same steps)
  int gend = 0;     // first step after the current data-symbol group
  if (producer) {
    // ================= producer: staging, conversion, first pass(es)
    StepCursor cur;   // next step to load
    cur.init(p);
    uint64_t pol = 0;
    if (warp == 0 && p.use_tma) {
      if (lane == 0) pol = evict_first_policy();
      pol = __shfl_sync(0xffffffffu, pol, 0);
    }
    float2 wpre[32];   // writer-side twiddles (N <= 1024)
    if constexpr (N <= 1024) writer_twiddles<LOG2N>(wpre, jt, tw);
    int issued = 0;    // steps whose copies warp 0 has issued (steps 0 .. issued-1)
    for (int g = 0; g < p.groups; ++g) {
      gend += p.chunks * group_items(p, g);
      // loads never run ahead into the next data-symbol group: its staging
      // ring holds the demapped codes at the end of each group; once a wait
      // has given up no copy is issued any more
      if (warp == 0 && p.use_tma && !*abort_flag) {
        fence_proxy_async();
        for (int i = step; i < step + K && i < gend; ++i) {
          issue_step<LOG2N, FC32>(p, f, cur.c, cur.symbol(p), stage + (i % K) * slot_bytes,
                                  lay.team_stage, smem_u32(&bars[i % K]), pol, lane);
          // test hook: the first staging phase of block 0 also waits for 16
          // bytes that no copy delivers, so its bounded wait runs out
          if (p.fault == 1 && blockIdx.x == 0 && i == 0 && lane == 0)
            mbar_expect_tx_only(smem_u32(&bars[0]), 16);
          cur.next(p);
          issued = i + 1;
        }
      }
      StepCursor me;    // the step this thread processes
      me.init(p);
      for (int i = 0; i < step; ++i) me.next(p);
      for (; step < gend; ++step, me.next(p)) {
        const int m = me.c * A + alpha;
        const bool valid = m < p.M;
        const int slot = step % K;
        float2 v[32];
        if (p.use_tma) {
          wait_slot(smem_u32(&bars[slot]), (step / K) & 1, abort_flag, p.status);
          if (valid) {
            load_row<LOG2N, FC32>(v, stage + slot * slot_bytes + alpha * lay.team_stage, jt, false);
          } else {
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
          }
        } else {
          if (valid) {
            load_row<LOG2N, FC32>(v, row_ptr<LOG2N, FC32>(p, f, m, me.symbol(p)), jt, true);
          } else {
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
          }
        }
        dft<32>(v, p);
        middle_pass<LOG2N>(v, ex1, jt, p.twP, p, [] { bar_sync(kBarProd, TW); });
        if constexpr (N <= 1024) {
#pragma unroll
          for (int k1 = 1; k1 < 32; ++k1) v[k1] = cmul(v[k1], wpre[k1]);
        }
        const int b = step & 1;
        if (step >= 2) bar_sync(kBarEmpty0 + b, T);   // consumers released buffer b
        final_exchange_write<LOG2N>(v, b ? ex0 + A * G::XS : ex0, jt);
        bar_arrive(kBarFull0 + b, T);
        bar_sync(kBarProd, TW);   // every producer is done with this staging slot
        if (warp == 0 && p.use_tma && step + K < gend && !*abort_flag) {
          fence_proxy_async();
          issue_step<LOG2N, FC32>(p, f, cur.c, cur.symbol(p), stage + slot * slot_bytes,
                                  lay.team_stage, smem_u32(&bars[slot]), pol, lane);
          cur.next(p);
          issued = step + K + 1;
        }
      }
      bar_sync(0, T);   // group's loop done (consumers finished too)
      bar_sync(0, T);   // consumers wrote the codes
      // pack: 8 consecutive subcarriers -> q bytes (producers and consumers)
      const int nd = min(p.dg, p.D - g * p.dg);
      const int items8 = (p.mode == kModePartial) ? 0 : nd * (N / 8);
      const size_t frame_bytes = static_cast<size_t>(p.D) * N * p.q / 8;
      const uint8_t* codes = smem + lay.codes_off;
      for (int it = tid; it < items8; it += T) {
        const int dl = it / (N / 8);
        const int k0 = (it % (N / 8)) * 8;
        uint64_t acc = 0;
#pragma unroll
        for (int bb = 0; bb < 8; ++bb) acc = (acc << p.q) | codes[dl * N + k0 + bb];
        uint8_t* dst = p.bits + f * frame_bytes + (static_cast<size_t>(g * p.dg + dl) * N + k0) * p.q / 8;
        for (int j = 0; j < p.q; ++j) dst[j] = static_cast<uint8_t>(acc >> (8 * (p.q - 1 - j)));
      }
      bar_sync(0, T);   // codes consumed before the ring is refilled
    }
    // balance the consumers' last two buffer releases
    if (step >= 2) bar_sync(kBarEmpty0 + (step & 1), T);
    if (step >= 1) bar_sync(kBarEmpty0 + ((step + 1) & 1), T);
    if (tid == 0 && p.use_tma && *abort_flag) {
      // a wait gave up: give any copy still in flight a bounded chance to
      // land (at most one per slot: the last K steps whose copies were issued)
      for (int s = 0; s < K && s < issued; ++s) {
        const int last = issued - 1 - ((issued - 1 - s) % K);
        (void)mbar_wait_bounded(smem_u32(&bars[last % K]), (last / K) & 1);
      }
    }
  } else {
    // ================= consumer: last pass, LS, MRC, accumulation, demap
    const uint32_t tacc = *tmem_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16);
    const uint32_t tE = tacc + 2 * OWN * p.dg;
    float zero[2 * OWN];
#pragma unroll
    for (int i = 0; i < 2 * OWN; ++i) zero[i] = 0.f;
    TmE::st(tE, zero);
    float2 h[32];
    float2 wlast[32];   // this thread's last-pass twiddles (N = 2048; the
                        // producer applies them itself for N <= 1024)
    if constexpr (N > 1024) final_twiddles<LOG2N>(wlast, jt, tw);
    for (int g = 0; g < p.groups; ++g) {
      const int nd = min(p.dg, p.D - g * p.dg);
      const int d0 = g * p.dg;
      for (int dl = 0; dl < nd; ++dl) TmP::st(tacc + 2 * OWN * dl, zero);
      const bool need_fft_pilot = fft_pilot(p) && g == 0;
      for (int c = 0; c < p.chunks; ++c) {
        const int m = c * A + alpha;
        const bool valid = m < p.M;
        const size_t hrow = (static_cast<size_t>(f) * p.Mtot + p.m0 + blockIdx.y * p.shard_y + m) * N;
        if (!need_fft_pilot) {
          // channel from memory: given (demodulate) or written in group 0
          const float2* Hs = fft_pilot(p) ? p.H_out : p.H_in;
#pragma unroll
          for (int e = 0; e < 32; ++e)
            h[e] = valid ? Hs[hrow + bin_of<LOG2N>(jt, e)] : make_float2(0.f, 0.f);
          if (g == 0) {
            // channel energy of this chunk: |H|^2 summed over its antennas
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
        const int items = group_items(p, g);
        for (int it = 0; it < items; ++it, ++step) {
          const bool is_pilot = need_fft_pilot && it == 0;
          const int d = d0 + it - (need_fft_pilot ? 1 : 0);
          const int b = step & 1;
          float2 v[32];
          bar_sync(kBarFull0 + b, T);
          if constexpr (N <= 1024) {
            final_exchange_read_plain<LOG2N>(v, b ? ex0 + A * G::XS : ex0, jt);
          } else {
            final_exchange_read_w<LOG2N>(v, b ? ex0 + A * G::XS : ex0, jt, wlast);
          }
          bar_arrive(kBarEmpty0 + b, T);
          final_dft<LOG2N>(v, p);
          if (is_pilot) {
            // LS estimate H = Y conj(X) / |X|^2 (1/sqrt(N) folded into xinv)
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int k = bin_of<LOG2N>(jt, e);
              const float2 hv = cmul(v[e], __ldg(p.xinv + k));
              h[e] = valid ? hv : make_float2(0.f, 0.f);
              if (valid) p.H_out[hrow + k] = hv;
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
            // MRC numerator: conj(H) Y summed over the antennas of the chunk
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = cmulc(h[e], v[e]);
            reduce_scatter<A, 16>(v, alpha);
            float acc[2 * OWN];
            const uint32_t tp = tacc + 2 * OWN * (d - d0);
            tmem_wait_st();
            TmP::ld(tp, acc);
            tmem_wait_ld();
#pragma unroll
            for (int cc = 0; cc < OWN; ++cc) {
              acc[2 * cc] += v[cc].x;
              acc[2 * cc + 1] += v[cc].y;
            }
            TmP::st(tp, acc);
          }
        }
      }
      tmem_wait_st();
      bar_sync(0, T);   // the group's steps are done; the staging ring is free
      uint8_t* codes = smem + lay.codes_off;
      if (p.mode == kModePartial) {
        // the shard's partial sums leave the block; the combine kernel forms
        // z over all shards (Y is the unscaled transform here: P gets the
        // unitary 1/sqrt(N), E is already a sum of unitary |H|^2)
        if (g == 0) {
          float e[OWN];
          TmE::ld(tE, e);
          tmem_wait_ld();
#pragma unroll
          for (int cc = 0; cc < OWN; ++cc)
            p.E_out[(static_cast<size_t>(blockIdx.y) * gridDim.x + f) * N +
                    bin_of<LOG2N>(jt, alpha * OWN + cc)] = e[cc];
        }
        for (int dl = 0; dl < nd; ++dl) {
          float acc[2 * OWN];
          TmP::ld(tacc + 2 * OWN * dl, acc);
          tmem_wait_ld();
          float2* dst = p.P_out + ((static_cast<size_t>(blockIdx.y) * gridDim.x + f) * p.D + d0 + dl) * N;
#pragma unroll
          for (int cc = 0; cc < OWN; ++cc)
            dst[bin_of<LOG2N>(jt, alpha * OWN + cc)] =
                make_float2(acc[2 * cc] * p.inv_sqrtN, acc[2 * cc + 1] * p.inv_sqrtN);
        }
      } else {
      float ie[OWN];
      if (g == 0) {
        float e[OWN];
        TmE::ld(tE, e);
        tmem_wait_ld();
        // E -> 1 / (sqrt(N) E); zero or non-finite energy flags the frame
#pragma unroll
        for (int cc = 0; cc < OWN; ++cc) {
          const bool ok = (e[cc] > 0.f) && (e[cc] <= 3.4028234663852886e38f);
          if (!ok) latch(p.status, kStDevice);
          ie[cc] = ok ? (1.0f / e[cc]) * p.inv_sqrtN : 0.f;
        }
        TmE::st(tE, ie);   // later data-symbol groups reuse 1/E
      } else {
        TmE::ld(tE, ie);
        tmem_wait_ld();
      }
      for (int dl = 0; dl < nd; ++dl) {
        float acc[2 * OWN];
        TmP::ld(tacc + 2 * OWN * dl, acc);
        tmem_wait_ld();
        const int d = d0 + dl;
#pragma unroll
        for (int cc = 0; cc < OWN; ++cc) {
          const int k = bin_of<LOG2N>(jt, alpha * OWN + cc);
          const float2 z = (ie[cc] != 0.f) ? make_float2(acc[2 * cc] * ie[cc], acc[2 * cc + 1] * ie[cc])
                                           : make_float2(0.f, 0.f);
          if (p.eq) p.eq[(static_cast<size_t>(f) * p.D + d) * N + k] = z;
          uint32_t code = gray(axis_level(z.x, p));
          if (p.axes == 2) code = (code << p.wbits) | gray(axis_level(z.y, p));
          codes[dl * N + k] = static_cast<uint8_t>(code);
        }
      }
      }
      tmem_wait_st();
      bar_sync(0, T);   // codes written
      // pack (shared with the producers)
      const int items8 = (p.mode == kModePartial) ? 0 : nd * (N / 8);
      const size_t frame_bytes = static_cast<size_t>(p.D) * N * p.q / 8;
      for (int it = tid; it < items8; it += T) {
        const int dl = it / (N / 8);
        const int k0 = (it % (N / 8)) * 8;
        uint64_t acc = 0;
#pragma unroll
        for (int bb = 0; bb < 8; ++bb) acc = (acc << p.q) | codes[dl * N + k0 + bb];
        uint8_t* dst = p.bits + f * frame_bytes + (static_cast<size_t>(d0 + dl) * N + k0) * p.q / 8;
        for (int j = 0; j < p.q; ++j) dst[j] = static_cast<uint8_t>(acc >> (8 * (p.q - 1 - j)));
      }
      bar_sync(0, T);
    }
    tmem_fence_before();
  }
  __syncthreads();
  tmem_fence_after();
  if (warp == W) tmem_dealloc(*tmem_base, p.tmem_cols);
}

// ======================================================= estimate kernel

// One warp group per block: antenna chunk c of frame f.
template <int LOG2N, bool FC32>
__global__ void __launch_bounds__(Geo<LOG2N>::TW) estimate_kernel(const KParams p) {
  using G = Geo<LOG2N>;
  constexpr int N = G::N, A = G::A, F = G::F;
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x / p.chunks;
  const int c = blockIdx.x % p.chunks;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int alpha = lane % A;
  const int jt = (tid >> 5) * F + lane / A;
  const Layout lay = make_layout(N, FC32 ? 8 : 4, 1, 1);
  const float2* tw = load_pass_twiddles<LOG2N>(p, smem, lay);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 192);
  unsigned char* stage = smem + lay.stage_off;
  float2* ex = reinterpret_cast<float2*>(smem + lay.ex_off) + alpha * G::XS;
  float2* ex1 = reinterpret_cast<float2*>(smem + lay.ex1_off) + alpha * G::XS;
  const int m = c * A + alpha;
  const bool valid = m < p.M;
  if (tid == 0) {
    *abort_flag = 0;
    if (p.use_tma) {
      mbar_init(smem_u32(&bars[0]), 1);
      fence_mbar_init();
    }
  }
  __syncthreads();
  if (tid < 32 && p.use_tma)
    issue_step<LOG2N, FC32>(p, f, c, p.pilot_idx, stage, lay.team_stage, smem_u32(&bars[0]),
                            evict_first_policy(), lane);
  float2 v[32];
  if (p.use_tma) wait_slot(smem_u32(&bars[0]), 0, abort_flag, p.status);
  if (valid) {
    if (p.use_tma)
      load_row<LOG2N, FC32>(v, stage + alpha * lay.team_stage, jt, false);
    else
      load_row<LOG2N, FC32>(v, row_ptr<LOG2N, FC32>(p, f, m, p.pilot_idx), jt, true);
  } else {
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
  }
  dft<32>(v, p);
  middle_pass<LOG2N>(v, ex1, jt, p.twP, p, [] { __syncthreads(); });
  final_exchange_write<LOG2N>(v, ex, jt);
  __syncthreads();
  final_exchange_read<LOG2N>(v, ex, jt, tw);
  final_dft<LOG2N>(v, p);
  if (valid) {
    const size_t hrow = (static_cast<size_t>(f) * p.Mtot + p.m0 + m) * N;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      const int k = bin_of<LOG2N>(jt, e);
      p.H_out[hrow + k] = cmul(v[e], __ldg(p.xinv + k));
    }
  }
}

// ======================================================= fft kernel

// One warp group per block: antenna chunk c of frame f, every symbol.
template <int LOG2N, bool FC32>
__global__ void __launch_bounds__(Geo<LOG2N>::TW) fft_kernel(const KParams p) {
  using G = Geo<LOG2N>;
  constexpr int N = G::N, A = G::A, F = G::F;
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x / p.chunks;
  const int c = blockIdx.x % p.chunks;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int alpha = lane % A;
  const int jt = (tid >> 5) * F + lane / A;
  const Layout lay = make_layout(N, FC32 ? 8 : 4, p.nslots, 1);
  const float2* tw = load_pass_twiddles<LOG2N>(p, smem, lay);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 192);
  unsigned char* stage = smem + lay.stage_off;
  float2* ex = reinterpret_cast<float2*>(smem + lay.ex_off) + alpha * G::XS;
  float2* ex1 = reinterpret_cast<float2*>(smem + lay.ex1_off) + alpha * G::XS;
  const int m = c * A + alpha;
  const bool valid = m < p.M;
  const int K = p.nslots;
  const int slot_bytes = A * lay.team_stage;
  uint64_t pol = 0;
  if (tid == 0) {
    *abort_flag = 0;
    if (p.use_tma) {
      for (int s = 0; s < K; ++s) mbar_init(smem_u32(&bars[s]), 1);
      fence_mbar_init();
    }
  }
  __syncthreads();
  if (tid < 32 && p.use_tma) {
    pol = evict_first_policy();
    for (int s = 0; s < K && s < p.S; ++s)
      issue_step<LOG2N, FC32>(p, f, c, s, stage + s * slot_bytes, lay.team_stage,
                              smem_u32(&bars[s]), pol, lane);
  }
  for (int s = 0; s < p.S; ++s) {
    const int slot = s % K;
    float2 v[32];
    if (p.use_tma) wait_slot(smem_u32(&bars[slot]), (s / K) & 1, abort_flag, p.status);
    if (valid) {
      if (p.use_tma)
        load_row<LOG2N, FC32>(v, stage + slot * slot_bytes + alpha * lay.team_stage, jt, false);
      else
        load_row<LOG2N, FC32>(v, row_ptr<LOG2N, FC32>(p, f, m, s), jt, true);
    } else {
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
    }
    dft<32>(v, p);
    __syncthreads();   // staging slot consumed; exchange buffers free
    if (tid < 32 && p.use_tma && s + K < p.S) {
      fence_proxy_async();
      issue_step<LOG2N, FC32>(p, f, c, s + K, stage + slot * slot_bytes, lay.team_stage,
                              smem_u32(&bars[slot]), pol, lane);
    }
    middle_pass<LOG2N>(v, ex1, jt, p.twP, p, [] { __syncthreads(); });
    final_exchange_write<LOG2N>(v, ex, jt);
    __syncthreads();
    final_exchange_read<LOG2N>(v, ex, jt, tw);
    final_dft<LOG2N>(v, p);
    if (valid) {
      float2* out = p.Y_out + ((static_cast<size_t>(f) * p.Mtot + p.m0 + m) * p.S + s) * N;
#pragma unroll
      for (int e = 0; e < 32; ++e)
        out[bin_of<LOG2N>(jt, e)] = make_float2(v[e].x * p.inv_sqrtN, v[e].y * p.inv_sqrtN);
    }
  }
}

#endif  // __CUDACC__

// Host-side launch entry of one FFT length (defined in lsas_inst_n*.cu).
using LaunchFn = cudaError_t (*)(int kind, bool fc32, const KParams& p, int grid,
                                 int smem, cudaStream_t st);
enum { kKindFrame = 0, kKindEstimate = 1, kKindFft = 2 };

}  // namespace lsas
