// lsas_kernels.cuh -- device code of liblsas for sm_103a.
//
// Three kernels share one building block, the "team FFT": a team of
// L = N/32 threads transforms one N-point OFDM symbol of one antenna, each
// thread holding 32 complex points in registers.  A Stockham auto-sort FFT
// (radix 32, then radix N/32; N = 2048 uses 32 x 8 x 8) runs its butterflies
// in registers and exchanges data between passes through a swizzled
// shared-memory buffer.  A block holds A teams = A antennas of one symbol.
//
// Input samples are staged by bulk asynchronous copies (cp.async.bulk, the
// TMA engine) into a ring of shared-memory slots, one contiguous CP-stripped
// symbol row per antenna, completion tracked by mbarriers; this is the CP
// removal of Sec. II-B done as addressing.  Every wait on an mbarrier is
// bounded: after ~2 s it latches LSAS_ERR_TIMEOUT and the block runs on
// without waiting again, so a missing completion can never hang the GPU.
//
//   frame_kernel    one block per frame: pilot FFT -> LS estimate H (kept in
//                   registers, written out) and the channel energy sum, then
//                   every data symbol: FFT -> conj(H) Y -> sum over antennas
//                   (shared-memory reduction) accumulated per subcarrier,
//                   then z = sum / energy -> Gray slicer -> packed bits.
//                   Sec. II-C (LS, MRC), Sec. III (conjugate and channel sum
//                   formed once and reused for every data symbol).
//   estimate_kernel one block per (frame, antenna chunk): pilot FFT -> H.
//   fft_kernel      one block per (frame, antenna chunk): all symbols -> Y.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lsas {

enum { kModeEstimate = 0, kModeDemod = 1, kModeRun = 2 };
enum { kStOk = 0, kStTimeout = 6, kStDevice = 7 };

constexpr int kMaxSlots = 4;
constexpr int kSmemHeader = 256;     // mbarriers (2 groups x 4 slots) + flags
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
  int M, S, cp, pilot_idx, D;
  int chunks;            // ceil(M / A)
  int groups, dg;        // data-symbol groups per frame, symbols per group
  int mode;              // kModeDemod or kModeRun (frame_kernel)
  int use_tma, nslots;
  int tmem_cols, tmem_cth;   // TMEM allocation (columns) and columns per thread
  int q, wbits, axes, nthr;
  float inv_sqrtN;
  float thr[kMaxThresholds];   // per-axis decision boundaries (float32)
  float2 w32[16];              // W_32^e = {cos, -sin}(2 pi e / 32), e < 16
  float2 w32n[16];             // {-Im, Re} of W_32^e (packed complex multiply)
};

// ---------------------------------------------------------------- geometry
//
// Thread mapping: a block holds G independent groups of W warps.  A warp's
// lanes hold A antennas x F = 32/A sub-lanes (antenna alpha = lane % A,
// sub-lane q = lane / A).  The FFT team of antenna alpha is the set of
// threads of one group with that alpha, team index jt = (warp in group) * F
// + q, L = W * F = N / 32 threads per team, 32 complex points per thread.
// Because the A antennas of one subcarrier sit in lanes of one warp, the sum
// over antennas of MRC is a warp-shuffle reduction, and lanes of different
// antennas share pass-twiddle loads.  The groups of a block process disjoint
// antenna chunks of the same frame with their own staging ring, exchange
// buffer, barriers and partial sums, so they run out of phase with each
// other; their partial sums are added in the demapping phase.

__host__ __device__ constexpr int geo_A(int N) { return N == 64 ? 16 : (N == 128 ? 8 : 4); }
__host__ __device__ constexpr int geo_G(int N) { return (N >= 256 && N <= 1024) ? 2 : 1; }
__host__ __device__ constexpr int geo_TG(int N) { return 32 * ((N / 32) / (32 / geo_A(N))); }
__host__ __device__ constexpr int geo_T(int N) { return geo_G(N) * geo_TG(N); }
// exchange stride (float2): N plus one pad per 32, then rounded so that
// antenna regions start 16/A float2 apart modulo the 16 bank pairs
__host__ __device__ constexpr int geo_XS(int N) {
  return (N + N / 32) + ((16 / geo_A(N) - (N + N / 32) % 16) + 16) % 16;
}
// staging stride pad (samples) per antenna: rows start F (sc16) or F/2
// (fc32) words of banks apart, and stay 16-byte aligned for bulk copies
__host__ __device__ constexpr int geo_spad(int N, int bps) {
  return bps == 4 ? ((32 / geo_A(N)) < 4 ? 4 : 32 / geo_A(N))
                  : ((16 / geo_A(N)) < 2 ? 2 : 16 / geo_A(N));
}

template <int LOG2N>
struct Geo {
  static constexpr int N = 1 << LOG2N;
  static constexpr int L = N / 32;          // threads per team
  static constexpr int A = geo_A(N);        // antennas per group step
  static constexpr int F = 32 / A;          // sub-lanes per warp
  static constexpr int W = L / F;           // warps per group
  static constexpr int TG = 32 * W;         // threads per group
  static constexpr int G = geo_G(N);        // groups per block (frame kernel)
  static constexpr int T = G * TG;          // threads per block (frame kernel)
  static constexpr int XS = geo_XS(N);
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Shared memory of a block: a header (mbarriers, flags, TMEM address), the
// pass twiddles, then one region per group: staging slots and exchange
// buffer.  After the chunk loop of the fused kernel, group 0's staging slots
// are reused for the partial-sum exchange between groups and for the
// demapped codes.
struct Layout {
  int tw_off;       // pass twiddles (float2[N], N <= 1024)
  int group_off;    // first group region
  int group_bytes;  // stride between group regions
  int team_stage;   // bytes per antenna per staging slot
  int stage_off;    // within a group region
  int ex_off;       // within a group region
  int merge_off;    // fused kernel: float2[2][N] partial sums + float[N] energy
  int codes_off;    // fused kernel: uint8[dg][N] demapped codes
  int total;
  int reuse_end;    // end of the reused region (must stay inside group 0's slots)
};

__host__ __device__ inline Layout make_layout(int N, int bps, int nslots, int dg, int groups,
                                              bool frame) {
  Layout l;
  const int A = geo_A(N);
  l.tw_off = kSmemHeader;
  l.group_off = align_up(l.tw_off + (N <= 1024 ? N * 8 : 0), 128);
  l.team_stage = (N + geo_spad(N, bps)) * bps;
  l.stage_off = 0;
  l.ex_off = align_up(nslots * A * l.team_stage, 128);
  l.group_bytes = align_up(l.ex_off + A * geo_XS(N) * 8, 128);
  l.total = l.group_off + groups * l.group_bytes;
  l.merge_off = l.group_off;
  l.codes_off = align_up(l.merge_off + (groups > 1 ? 2 * N * 8 + N * 4 : 0), 128);
  l.reuse_end = frame ? l.codes_off + dg * N : l.group_off;
  return l;
}

// Per-thread accumulators of the fused kernel live in tensor memory (TMEM):
// OWN = 32/A subcarriers per thread after the antenna reduction, for dg data
// symbols (complex) plus the channel energy.  Warps sharing a TMEM lane
// quarter (warp % 4) split the columns by warp / 4.
__host__ __device__ constexpr int geo_OWN(int N) { return 32 / geo_A(N); }
__host__ __device__ inline int tmem_cols_thread(int N, int dg) {
  return 2 * geo_OWN(N) * dg + geo_OWN(N);
}
__host__ __device__ inline int tmem_warps_per_quarter(int N) {
  return geo_T(N) / 32 > 4 ? geo_T(N) / 128 : 1;
}
__host__ __device__ inline int tmem_alloc_cols(int N, int dg) {
  const int need = tmem_cols_thread(N, dg) * tmem_warps_per_quarter(N);
  int c = 32;
  while (c < need) c *= 2;
  return c;
}

// Number of pass twiddles in the host-built table (layout in pass_twiddles):
// N <= 1024: [r][j] = W_N^(j r), r < N/32, j < 32 (second pass);
// N = 2048:  [r][j] = W_2048^(8 j r), j < 32 (second pass), then
//            [256 + r*256 + j] = W_2048^(j r), j < 256 (third pass).
__host__ __device__ inline int pass_tw_count(int N) { return N <= 1024 ? N : 256 + 2048; }

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
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src,
                                          uint32_t bytes, uint32_t bar,
                                          uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
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

// b * W_32^e for a compile-time e in [0, 16)
__device__ __forceinline__ float2 tw32(float2 b, int e, const KParams& p) {
  constexpr float kS = 0.70710678118654752440f;  // 1/sqrt(2)
  if (e == 0) return b;
  if (e == 8) return make_float2(b.y, -b.x);                                     // -j
  if (e == 4) return __fmul2_rn(make_float2(b.x + b.y, b.y - b.x), make_float2(kS, kS));
  if (e == 12) return __fmul2_rn(make_float2(b.y - b.x, -(b.x + b.y)), make_float2(kS, kS));
  return cmulw(b, p.w32[e], p.w32n[e]);
}

// One radix-2 decimation-in-time stage of half-span S on R registers.
template <int R, int S>
__device__ __forceinline__ void dit_stage(float2* a, const KParams& p) {
#pragma unroll
  for (int base = 0; base < R; base += 2 * S) {
#pragma unroll
    for (int i = 0; i < S; ++i) {
      const float2 b = tw32(a[base + i + S], i * (16 / S), p);
      const float2 x = a[base + i];
      a[base + i] = cadd(x, b);
      a[base + i + S] = csub(x, b);
    }
  }
}
template <int R, int S>
__device__ __forceinline__ void dit_stages(float2* a, const KParams& p) {
  if constexpr (S < R) {
    dit_stage<R, S>(a, p);
    dit_stages<R, 2 * S>(a, p);
  }
}

// In-register R-point DFT (R <= 32), natural order in and out: radix-2
// decimation in time over bit-reversed register indices (free renaming).
template <int R>
__device__ __forceinline__ void dft(float2* v, const KParams& p) {
  constexpr int LOGR = ilog2c(R);
  float2 a[R];
#pragma unroll
  for (int i = 0; i < R; ++i) a[i] = v[brev(i, LOGR)];
  dit_stages<R, 1>(a, p);
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = a[i];
}

// Padded exchange index: one float2 of padding after every 32 entries, so
// that both the row writes (t*32 + r) and the column reads (j + 32 r) of a
// transpose hit distinct banks, and every address is a per-thread base plus
// a compile-time offset.
__device__ __forceinline__ int xpad(int n) { return n + (n >> 5); }

// Synchronise one FFT team's group (gi): a warp, a named barrier, or the block.
template <int LOG2N>
__device__ __forceinline__ void team_sync(int gi) {
  using G = Geo<LOG2N>;
  if constexpr (G::W == 1) {
    __syncwarp();
  } else if constexpr (G::G == 1) {
    __syncthreads();
  } else {
    named_sync(1 + gi, G::TG);
  }
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

// Owner of bin k after the antenna reduction: the group thread (tid) whose
// register e = alpha * (32/A) + c holds it, and the slot c.  Inverse of
// bin_of with the thread mapping of Geo.
template <int LOG2N>
__device__ __forceinline__ void owner_of(int k, int& tid, int& c) {
  using G = Geo<LOG2N>;
  constexpr int OWN = 32 / G::A;
  int jt, e;
  if constexpr (G::N <= 1024) {
    const int kl = k & 31;
    jt = kl % G::L;
    e = (kl / G::L) * G::L + (k >> 5);
  } else {
    jt = k & 63;
    e = 8 * ((k >> 6) & 3) + (k >> 8);
  }
  const int alpha = e / OWN;
  c = e % OWN;
  tid = (jt / G::F) * 32 + (jt % G::F) * G::A + alpha;
}

// One interleaved int16 IQ word -> {I, Q} as floats, exactly, without the
// conversion unit: flipping the sign bits gives offset-binary u = v + 32768,
// 0x4B000000 | u is the float 2^23 + u, and one packed subtraction of
// 2^23 + 32768 leaves v.
__device__ __forceinline__ float2 sc16_to_float2(uint32_t w) {
  const uint32_t u = w ^ 0x80008000u;
  const uint32_t lo = (u & 0xffffu) | 0x4b000000u;
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

// Remaining FFT passes: v holds the radix-32 pass-1 outputs of team thread
// jt (Y1[jt*32 + r]); on return v[e] = Y[bin_of(jt, e)] (unscaled).  ex is
// this antenna's exchange region; tw the pass twiddles (shared memory for
// N <= 1024, global for N = 2048).  Every thread of the block calls this.
template <int LOG2N, typename AfterSync>
__device__ __forceinline__ void team_fft_rest(float2 (&v)[32], float2* ex, int jt, int gi,
                                              const float2* tw, const KParams& p,
                                              AfterSync&& after_sync) {
  using G = Geo<LOG2N>;
  constexpr int L = G::L;
#pragma unroll
  for (int r = 0; r < 32; ++r) ex[xpad(jt * 32 + r)] = v[r];
  team_sync<LOG2N>(gi);
  after_sync();   // work placed where the team does not wait on it
  if constexpr (G::N <= 1024) {
#pragma unroll
    for (int i = 0; i < 32 / L; ++i) {
      const int j = jt + i * L;
#pragma unroll
      for (int r = 0; r < L; ++r) {
        const float2 u = ex[xpad(j + 32 * r)];
        if (r == 0) {
          v[i * L + r] = u;
        } else {
          v[i * L + r] = cmul(u, tw[r * 32 + j]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 32 / L; ++i) dft<L>(v + i * L, p);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = jt + 64 * i;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float2 u = ex[xpad(j + 256 * r)];
        if (r == 0) {
          v[i * 8 + r] = u;
        } else {
          v[i * 8 + r] = cmul(u, __ldg(tw + r * 32 + (j & 31)));
        }
      }
    }
    team_sync<LOG2N>(gi);   // all reads done before the second exchange
#pragma unroll
    for (int i = 0; i < 4; ++i) dft<8>(v + i * 8, p);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = jt + 64 * i;
#pragma unroll
      for (int r = 0; r < 8; ++r) ex[xpad((j >> 5) * 256 + (j & 31) + 32 * r)] = v[i * 8 + r];
    }
    team_sync<LOG2N>(gi);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = jt + 64 * i;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float2 u = ex[xpad(j + 256 * r)];
        if (r == 0) {
          v[i * 8 + r] = u;
        } else {
          v[i * 8 + r] = cmul(u, __ldg(tw + 256 + r * 256 + j));
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) dft<8>(v + i * 8, p);
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

// Pass twiddles for the block: copied to shared memory when N <= 1024.
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

// ------------------------------------------------------- staging pipeline

// Items per antenna chunk in data-symbol group g: the pilot first (group 0 of
// the fused mode), then the group's data symbols.
__device__ __forceinline__ int group_items(const KParams& p, int g) {
  const int nd = min(p.dg, p.D - g * p.dg);
  return nd + ((p.mode == kModeRun && g == 0) ? 1 : 0);
}
// Antenna chunks handled by block group gi of G: c = gi, gi + G, ...
__device__ __forceinline__ int chunks_of(const KParams& p, int gi, int G) {
  return (p.chunks - gi + G - 1) / G;
}
template <int LOG2N, bool FC32>
__device__ __forceinline__ const unsigned char* row_ptr(const KParams& p, int f, int m,
                                                        int s) {
  constexpr int bps = FC32 ? 8 : 4;
  const size_t row = (static_cast<size_t>(f) * p.M + m) * p.S + s;
  return static_cast<const unsigned char*>(p.in) +
         (row * (Geo<LOG2N>::N + p.cp) + p.cp) * bps;
}

// Issue the bulk copies of one step (antennas of chunk c, symbol s) into a
// slot.  Called by a whole warp: lane 0 registers the byte count on the
// slot's mbarrier and lane a issues the copy of antenna row a.
template <int LOG2N, bool FC32>
__device__ __forceinline__ void issue_step(const KParams& p, int f, int c, int s,
                                           unsigned char* slot, int team_stage,
                                           uint32_t bar, uint64_t pol, int lane) {
  using G = Geo<LOG2N>;
  constexpr uint32_t bytes = G::N * (FC32 ? 8 : 4);
  const int nvalid = min(G::A, p.M - c * G::A);
  if (lane == 0) mbar_expect_tx(bar, bytes * nvalid);
  if (lane < nvalid)
    bulk_load(smem_u32(slot + lane * team_stage), row_ptr<LOG2N, FC32>(p, f, c * G::A + lane, s),
              bytes, bar, pol);
}

// Walks the steps of one block group in order (data-symbol group, chunk,
// item) with O(1) work per step.
struct StepCursor {
  int g, u, it, items, nc, G, gi;
  __device__ void init(const KParams& p, int gi_, int G_) {
    gi = gi_;
    G = G_;
    nc = chunks_of(p, gi, G);
    g = 0;
    u = 0;
    it = 0;
    items = group_items(p, 0);
  }
  // chunk and symbol of the current step
  __device__ int chunk() const { return gi + G * u; }
  __device__ int symbol(const KParams& p) const {
    int i = it;
    if (p.mode == kModeRun && g == 0) {
      if (i == 0) return p.pilot_idx;
      --i;
    }
    const int d = g * p.dg + i;
    return d < p.pilot_idx ? d : d + 1;
  }
  __device__ void next(const KParams& p) {
    if (++it < items) return;
    it = 0;
    if (++u < nc) return;
    u = 0;
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
  if (*abort_flag) return;
  if (!mbar_wait_bounded(bar, parity)) {
    *abort_flag = 1;
    latch(status, kStTimeout);
  }
}

// Level of one axis value: boundaries at or below v (ties go up).
__device__ __forceinline__ int axis_level(float v, const KParams& p) {
  int l = 0;
#pragma unroll
  for (int b = 0; b < kMaxThresholds; ++b)
    if (b < p.nthr) l += (v >= p.thr[b]) ? 1 : 0;
  return l;
}
__device__ __forceinline__ uint32_t gray(int l) { return static_cast<uint32_t>(l ^ (l >> 1)); }

// ======================================================= frame kernel

template <int LOG2N, bool FC32>
__global__ void __launch_bounds__(Geo<LOG2N>::T, 1) frame_kernel(const KParams p) {
  using G = Geo<LOG2N>;
  constexpr int N = G::N, A = G::A, T = G::T, TG = G::TG, F = G::F, NG = G::G;
  constexpr int OWN = 32 / A;  // subcarriers per thread after the antenna reduction
  using TmP = Tmem<2 * OWN>;   // one data symbol of partial sums (complex)
  using TmE = Tmem<OWN>;       // channel energy
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int gi = tid / TG;             // group of this thread
  const int ltid = tid % TG;           // thread index within the group
  const int lane = tid & 31;
  const int alpha = lane % A;
  const int jt = (ltid >> 5) * F + lane / A;
  const Layout lay = make_layout(N, FC32 ? 8 : 4, p.nslots, p.dg, NG, true);
  const float2* tw = load_pass_twiddles<LOG2N>(p, smem, lay);
  const int K = p.nslots;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem) + gi * kMaxSlots;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 192 + 4 * gi);
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(smem + 160);
  unsigned char* greg = smem + lay.group_off + gi * lay.group_bytes;
  unsigned char* stage = greg + lay.stage_off;
  float2* myex = reinterpret_cast<float2*>(greg + lay.ex_off) + alpha * G::XS;
  const int slot_bytes = A * lay.team_stage;
  const int nc = chunks_of(p, gi, NG);

  int total = 0;
  for (int g = 0; g < p.groups; ++g) total += nc * group_items(p, g);

  uint64_t pol = 0;
  if (ltid == 0) {
    *abort_flag = 0;
    if (p.use_tma) {
      for (int s = 0; s < K; ++s) mbar_init(smem_u32(&bars[s]), 1);
      fence_mbar_init();
    }
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_base), p.tmem_cols);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  // this thread's TMEM lane and first column: P(dl) at 2*OWN*dl, E after the dg symbols
  const uint32_t tacc = *tmem_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                        static_cast<uint32_t>((warp >> 2) * p.tmem_cth);
  const uint32_t tE = tacc + 2 * OWN * p.dg;

  StepCursor cur;   // next step to load (meaningful in warp 0 of the group)
  cur.init(p, gi, NG);
  if (ltid < 32 && p.use_tma) {
    if (ltid == 0) pol = evict_first_policy();
    pol = __shfl_sync(0xffffffffu, pol, 0);
  }

  float zero[2 * OWN];
#pragma unroll
  for (int i = 0; i < 2 * OWN; ++i) zero[i] = 0.f;
  TmE::st(tE, zero);

  float2 h[32];
  int step = 0;
  int gend = 0;   // first step after the current data-symbol group
  for (int g = 0; g < p.groups; ++g) {
    const int nd = min(p.dg, p.D - g * p.dg);
    const int d0 = g * p.dg;
    for (int dl = 0; dl < nd; ++dl) TmP::st(tacc + 2 * OWN * dl, zero);
    // loads never run ahead into the next data-symbol group: group 0's
    // staging slots are reused by the demap phase at its end
    gend += nc * group_items(p, g);
    if (ltid < 32 && p.use_tma) {
      fence_proxy_async();   // the demap phase wrote these slots through the generic proxy
      for (int i = step; i < step + K && i < gend; ++i) {
        issue_step<LOG2N, FC32>(p, f, cur.chunk(), cur.symbol(p), stage + (i % K) * slot_bytes,
                                lay.team_stage, smem_u32(&bars[i % K]), pol, lane);
        cur.next(p);
      }
    }

    for (int u = 0; u < nc; ++u) {
      const int c = gi + NG * u;
      const int m = c * A + alpha;
      const bool valid = m < p.M;
      const size_t hrow = (static_cast<size_t>(f) * p.M + m) * N;
      const bool need_fft_pilot = (p.mode == kModeRun && g == 0);
      if (!need_fft_pilot) {
        // channel from memory: given (demodulate) or written in group 0
        const float2* Hs = (p.mode == kModeRun) ? p.H_out : p.H_in;
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
        const int s = is_pilot ? p.pilot_idx : (d < p.pilot_idx ? d : d + 1);
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
            load_row<LOG2N, FC32>(v, row_ptr<LOG2N, FC32>(p, f, m, s), jt, true);
          } else {
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
          }
        }
        dft<32>(v, p);
        team_sync<LOG2N>(gi);  // staging slot consumed; exchange buffer free
        // refill the consumed slot once the exchange barrier has passed, so
        // the other warps of the group do not wait on the issuing warp
        team_fft_rest<LOG2N>(v, myex, jt, gi, tw, p, [&] {
          if (ltid < 32 && p.use_tma && step + K < gend) {
            fence_proxy_async();
            issue_step<LOG2N, FC32>(p, f, cur.chunk(), cur.symbol(p), stage + slot * slot_bytes,
                                    lay.team_stage, smem_u32(&bars[slot]), pol, lane);
            cur.next(p);
          }
        });
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
    // ---- demap: owners read their sums from TMEM; with two groups the
    // partner group's partial sums come through shared memory
    tmem_wait_st();
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    float2* mP = reinterpret_cast<float2*>(smem + lay.merge_off);   // [2][N]
    float* mE = reinterpret_cast<float*>(smem + lay.merge_off + 2 * N * 8);
    uint8_t* codes = smem + lay.codes_off;
    float ie[OWN];
    if (g == 0) {
      float e[OWN];
      TmE::ld(tE, e);
      tmem_wait_ld();
      if constexpr (NG > 1) {
        if (gi == 1) {
#pragma unroll
          for (int cc = 0; cc < OWN; ++cc) mE[cc * TG + ltid] = e[cc];
        }
        __syncthreads();
        if (gi == 0) {
#pragma unroll
          for (int cc = 0; cc < OWN; ++cc) {
            e[cc] += mE[cc * TG + ltid];
            mE[cc * TG + ltid] = e[cc];
          }
        }
        __syncthreads();
        if (gi == 1) {
#pragma unroll
          for (int cc = 0; cc < OWN; ++cc) e[cc] = mE[cc * TG + ltid];
        }
      }
      // E -> 1 / (sqrt(N) E); zero or non-finite energy flags the frame
#pragma unroll
      for (int cc = 0; cc < OWN; ++cc) {
        const bool ok = (e[cc] > 0.f) && (e[cc] <= 3.4028234663852886e38f);
        if (!ok) latch(p.status, kStDevice);
        ie[cc] = ok ? (1.0f / e[cc]) * p.inv_sqrtN : 0.f;
      }
      // keep 1/E in the energy columns for the later data-symbol groups
      TmE::st(tE, ie);
    } else {
      TmE::ld(tE, ie);
      tmem_wait_ld();
    }
    // symbols are demapped in pairs: group q takes the symbol of parity q
    for (int dl0 = 0; dl0 < nd; dl0 += NG) {
      const int dl = dl0 + gi;            // symbol this thread demaps
      float acc[2 * OWN];
      if constexpr (NG > 1) {
        // hand the partner group the partial sums of its symbol
        const int dp = dl0 + (1 - gi);
        if (dp < nd) {
          TmP::ld(tacc + 2 * OWN * dp, acc);
          tmem_wait_ld();
#pragma unroll
          for (int cc = 0; cc < OWN; ++cc)
            mP[(1 - gi) * N + cc * TG + ltid] = make_float2(acc[2 * cc], acc[2 * cc + 1]);
        }
        __syncthreads();
      }
      if (dl < nd) {
        TmP::ld(tacc + 2 * OWN * dl, acc);
        tmem_wait_ld();
        const int d = d0 + dl;
#pragma unroll
        for (int cc = 0; cc < OWN; ++cc) {
          float2 sum = make_float2(acc[2 * cc], acc[2 * cc + 1]);
          if constexpr (NG > 1) sum = cadd(sum, mP[gi * N + cc * TG + ltid]);
          const int k = bin_of<LOG2N>(jt, alpha * OWN + cc);
          const float2 z = (ie[cc] != 0.f) ? make_float2(sum.x * ie[cc], sum.y * ie[cc])
                                           : make_float2(0.f, 0.f);
          if (p.eq) p.eq[(static_cast<size_t>(f) * p.D + d) * N + k] = z;
          uint32_t code = gray(axis_level(z.x, p));
          if (p.axes == 2) code = (code << p.wbits) | gray(axis_level(z.y, p));
          codes[dl * N + k] = static_cast<uint8_t>(code);
        }
      }
      if constexpr (NG > 1) __syncthreads();
    }
    __syncthreads();
    // pack: 8 consecutive subcarriers -> q bytes
    const int items8 = nd * (N / 8);
    const size_t frame_bytes = static_cast<size_t>(p.D) * N * p.q / 8;
    for (int it = tid; it < items8; it += T) {
      const int dl = it / (N / 8);
      const int k0 = (it % (N / 8)) * 8;
      uint64_t acc = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) acc = (acc << p.q) | codes[dl * N + k0 + b];
      uint8_t* dst = p.bits + f * frame_bytes + (static_cast<size_t>(d0 + dl) * N + k0) * p.q / 8;
      for (int j = 0; j < p.q; ++j) dst[j] = static_cast<uint8_t>(acc >> (8 * (p.q - 1 - j)));
    }
    tmem_wait_st();
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
  }
  if (ltid == 0 && p.use_tma && *abort_flag) {
    // a wait gave up: give any copy still in flight a bounded chance to land
    for (int s = 0; s < K && s < total; ++s) {
      const int last = total - 1 - ((total - 1 - s) % K);
      (void)mbar_wait_bounded(smem_u32(&bars[last % K]), (last / K) & 1);
    }
  }
  if (warp == 0) tmem_dealloc(*tmem_base, p.tmem_cols);
}

// ======================================================= estimate kernel

// One group per block: antenna chunk c of frame f.
template <int LOG2N, bool FC32>
__global__ void __launch_bounds__(Geo<LOG2N>::TG) estimate_kernel(const KParams p) {
  using G = Geo<LOG2N>;
  constexpr int N = G::N, A = G::A, F = G::F;
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x / p.chunks;
  const int c = blockIdx.x % p.chunks;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int alpha = lane % A;
  const int jt = (tid >> 5) * F + lane / A;
  const Layout lay = make_layout(N, FC32 ? 8 : 4, 1, 0, 1, false);
  const float2* tw = load_pass_twiddles<LOG2N>(p, smem, lay);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 192);
  unsigned char* stage = smem + lay.group_off + lay.stage_off;
  float2* myex = reinterpret_cast<float2*>(smem + lay.group_off + lay.ex_off) + alpha * G::XS;
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
  team_fft_rest<LOG2N>(v, myex, jt, 0, tw, p, [] {});
  if (valid) {
    const size_t hrow = (static_cast<size_t>(f) * p.M + m) * N;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      const int k = bin_of<LOG2N>(jt, e);
      p.H_out[hrow + k] = cmul(v[e], __ldg(p.xinv + k));
    }
  }
}

// ======================================================= fft kernel

// One group per block: antenna chunk c of frame f, every symbol.
template <int LOG2N, bool FC32>
__global__ void __launch_bounds__(Geo<LOG2N>::TG) fft_kernel(const KParams p) {
  using G = Geo<LOG2N>;
  constexpr int N = G::N, A = G::A, F = G::F;
  extern __shared__ __align__(128) unsigned char smem[];
  const int f = blockIdx.x / p.chunks;
  const int c = blockIdx.x % p.chunks;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int alpha = lane % A;
  const int jt = (tid >> 5) * F + lane / A;
  const Layout lay = make_layout(N, FC32 ? 8 : 4, p.nslots, 0, 1, false);
  const float2* tw = load_pass_twiddles<LOG2N>(p, smem, lay);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 192);
  unsigned char* stage = smem + lay.group_off + lay.stage_off;
  float2* myex = reinterpret_cast<float2*>(smem + lay.group_off + lay.ex_off) + alpha * G::XS;
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
    __syncthreads();
    team_fft_rest<LOG2N>(v, myex, jt, 0, tw, p, [&] {
      if (tid < 32 && p.use_tma && s + K < p.S) {
        fence_proxy_async();
        issue_step<LOG2N, FC32>(p, f, c, s + K, stage + slot * slot_bytes, lay.team_stage,
                                smem_u32(&bars[slot]), pol, lane);
      }
    });
    if (valid) {
      float2* out = p.Y_out + ((static_cast<size_t>(f) * p.M + m) * p.S + s) * N;
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
