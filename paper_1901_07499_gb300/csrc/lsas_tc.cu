// lsas_tc.cu -- the FFT of Sec. II-C as tensor-core DFT-factor GEMMs, and a
// staged LS / MRC / demap pass that reads the transformed symbols from memory.
//
// Tensor-core FFT (N = 32 N2, N2 = N/32 in {16, 32, 64}).  With n = N2 n1 + n2
// and k = k1 + 32 k2,
//   stage 1   A1[n2][k1] = sum_n1 x[N2 n1 + n2] W_32^(n1 k1)        (GEMM, K = 32)
//   twiddle   B1[n2][k1] = A1[n2][k1] W_N^(n2 k1)
//   stage 2   X[k1 + 32 k2] = sum_n2 B1[n2][k1] W_N2^(n2 k2)       (GEMM, K = N2)
// Each complex GEMM is a real one over [re | im] halves: a data row is
// [x_re(0..K-1) | x_im(0..K-1)] and the DFT operand row of output (re, k) is
// [cos | sin], of (im, k) [-sin | cos] (angle 2 pi n k / K).  Operands are
// fp16 or bf16 (both of one type in an MMA), accumulators fp32 in tensor
// memory (tcgen05.mma kind::f16, M = 128).  With terms = 3 every operand is
// split into hi = round(v) and lo = round(v - hi), and
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (the lo*lo term is dropped: ~2^-22
// relative for fp16, ~2^-16 for bf16); terms = 1 uses a_hi b_hi alone
// (~2^-11 relative for fp16, ~2^-8 for bf16).  Stage-2 inputs are scaled by 2^-6 (exact) to stay in
// fp16 range; the output is scaled back with the unitary 1/sqrt(N).
//
// Operand tiles use the canonical no-swizzle K-major layout (8-row x 16-byte
// core matrices, adjacent along K at 128 B, row groups at 128 * K / 8 B),
// except the stage-2 data operand, which the twiddle phase writes MN-major
// (8 rows contiguous): each thread holds one of its columns, so no transpose
// buffer is needed between the stages.
#include <cfloat>
#include <cmath>
#include <vector>

#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lsas_kernels.cuh"

namespace lsas {

// threads per block: 128 (one per operand row), or 256 for N = 2048, where
// two threads share each row of the twiddle, stage-2 and output phases
// (halves of the columns) and one batch's phases are the critical path
template <int LOG2N>
__host__ __device__ constexpr int tc_threads() { return LOG2N == 11 ? 256 : 128; }

// byte offset of element (row, k) of a rows x K fp16 operand tile
__host__ __device__ inline int tc_off(int row, int k, int K) {
  return (row >> 3) * (16 * K) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
// byte offset of element (row, k) of a 128-row MN-major operand tile: 8 rows
// contiguous (16 B), then 8 columns of them (a 128 B core matrix), the 16
// row groups of a column group 128 B apart, column groups 2048 B apart
__host__ __device__ inline int tc_mn_off(int row, int k) {
  return (row >> 3) * 128 + (k >> 3) * 2048 + (k & 7) * 16 + (row & 7) * 2;
}

// bfloat16 of a double, round to nearest even, by way of float
static uint16_t bf16_bits(double v) {
  const float f = static_cast<float>(v);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(u >> 16);
}
static double bf16_value(uint16_t b) {
  const uint32_t u = static_cast<uint32_t>(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Host: operand images of the K-point DFT, 2K rows x 2K columns: fp16 hi and
// lo, then bf16 hi and lo (each image 2K x 2K halves, in that order).
static void dft_image(int K, std::vector<uint16_t>& img) {
  const int R = 2 * K, C = 2 * K;
  img.assign(4 * R * C, 0);
  for (int r = 0; r < R; ++r) {
    const int k = r % K;
    for (int c = 0; c < C; ++c) {
      const int n = c % K;
      const double a = 2.0 * M_PI * static_cast<double>((static_cast<long>(n) * k) % K) / K;
      // out re: x_re cos + x_im sin; out im: -x_re sin + x_im cos
      const double w = (r < K) ? (c < K ? std::cos(a) : std::sin(a))
                               : (c < K ? -std::sin(a) : std::cos(a));
      const __half hi = __double2half(w);
      const __half lo = __double2half(w - static_cast<double>(__half2float(hi)));
      const uint16_t bhi = bf16_bits(w);
      const uint16_t blo = bf16_bits(w - bf16_value(bhi));
      const int o = tc_off(r, c, C) / 2;
      img[o] = __half_as_ushort(hi);
      img[R * C + o] = __half_as_ushort(lo);
      img[2 * R * C + o] = bhi;
      img[3 * R * C + o] = blo;
    }
  }
}

// Tables of the tensor-core FFT for one N (host side; the plan uploads them).
bool tc_tables(int N, std::vector<uint16_t>& w1, std::vector<uint16_t>& w2,
               std::vector<float2>& tw) {
  const int N2 = N / 32;
  if (N2 < 16 || N2 > 64) return false;
  dft_image(32, w1);
  dft_image(N2, w2);
  tw.resize(static_cast<size_t>(N2) * 32);
  for (int n2 = 0; n2 < N2; ++n2)
    for (int k1 = 0; k1 < 32; ++k1) {
      const double a = -2.0 * M_PI * static_cast<double>((n2 * k1) % N) / N;
      tw[n2 * 32 + k1] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
    }
  return true;
}

// ---------------------------------------------------------------- device

// Operand images are K-major rows of K halves: core matrices adjacent along K
// are 128 bytes apart, 8-row groups 16 K bytes apart.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, int K) { return umma_desc(addr, 128, 16 * K); }

// (a, b) -> packed fp16 hi = fp16(v) and lo = fp16(v - hi), as 32-bit words
__device__ __forceinline__ void split16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}
// the same with bf16 pieces: hi = bf16(v), lo = bf16(v - hi)
__device__ __forceinline__ void splitbf16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Store columns [C0, C1) of one operand row of 2K values (re[0..K) then
// im[0..K)), hi and lo images, in fp16 or bf16.
template <int K, int C0 = 0, int C1 = 2 * K>
__device__ __forceinline__ void store_row(unsigned char* hi_img, unsigned char* lo_img, int row,
                                          const float* re, const float* im, bool want_lo,
                                          bool bf16) {
#pragma unroll
  for (int c = C0; c < C1; c += 8) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const float a = c + j < K ? re[c + j] : im[c + j - K];
      const float b = c + j + 1 < K ? re[c + j + 1] : im[c + j + 1 - K];
      if (bf16) splitbf16x2(a, b, h[j / 2], l[j / 2]);
      else split16x2(a, b, h[j / 2], l[j / 2]);
    }
    const int o = tc_off(row, c, 2 * K);
    *reinterpret_cast<uint4*>(hi_img + o) = make_uint4(h[0], h[1], h[2], h[3]);
    if (want_lo) *reinterpret_cast<uint4*>(lo_img + o) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

template <int LOG2N>
struct TcGeo {
  static constexpr int N = 1 << LOG2N;
  static constexpr int N2 = N / 32;
  static constexpr int R = (128 / N2 > 4) ? 128 / N2 : 4;   // antenna-symbols per batch
  static constexpr int T1 = R * N2 / 128;                   // stage-1 tiles of 128 rows
  static constexpr int T2 = R * 32 / 128;                   // stage-2 tiles
  static constexpr int W1_BYTES = 64 * 64 * 2;              // one image
  static constexpr int W2_BYTES = (2 * N2) * (2 * N2) * 2;
  static constexpr int A1_BYTES = 128 * 64 * 2;             // one tile, one image
  static constexpr int A2_BYTES = 128 * (2 * N2) * 2;
  static constexpr int OFF_W1 = 0;
  static constexpr int OFF_W2 = OFF_W1 + 2 * W1_BYTES;
  static constexpr int OFF_A1 = OFF_W2 + 2 * W2_BYTES;      // A1 tiles [tile][hi, lo]
  static constexpr int A1_REGION = 2 * T1 * A1_BYTES;
  static constexpr int OFF_A2 = OFF_A1 + A1_REGION;
  static constexpr int OFF_BAR = OFF_A2 + 2 * T2 * A2_BYTES;
  static constexpr int SMEM = OFF_BAR + 64;
  static constexpr int TT = tc_threads<LOG2N>();            // threads per block
  static constexpr int PARTS = TT / 128;                    // threads per operand row
  static_assert(PARTS == 1 || T2 == 1, "two threads per row need one stage-2 tile");
};

// Tensor-core FFT: p.nframes rows of N samples (antenna-symbols, CP dropped)
// -> Y rows (unitary).  Persistent: block b takes batches b, b + grid, ...
template <int LOG2N, bool FC32>
__global__ void __launch_bounds__(tc_threads<LOG2N>(), 1) tcfft_kernel(const KParams p) {
  using G = TcGeo<LOG2N>;
  constexpr int N = G::N, N2 = G::N2, R = G::R, TT = G::TT, PARTS = G::PARTS;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const bool split = p.terms == 3;
  const bool bf16 = p.tc_bf16 != 0;
  unsigned char* w1 = smem + G::OFF_W1;
  unsigned char* w2 = smem + G::OFF_W2;
  unsigned char* a1 = smem + G::OFF_A1;
  unsigned char* a2 = smem + G::OFF_A2;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + G::OFF_BAR);
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(smem + G::OFF_BAR + 16);
  // constant DFT operands (hi, lo of the operand type) into shared memory
  {
    const uint4* s1 = static_cast<const uint4*>(p.tc_w1) + (bf16 ? 2 * G::W1_BYTES / 16 : 0);
    const uint4* s2 = static_cast<const uint4*>(p.tc_w2) + (bf16 ? 2 * G::W2_BYTES / 16 : 0);
    for (int i = tid; i < 2 * G::W1_BYTES / 16; i += TT) reinterpret_cast<uint4*>(w1)[i] = s1[i];
    for (int i = tid; i < 2 * G::W2_BYTES / 16; i += TT) reinterpret_cast<uint4*>(w2)[i] = s2[i];
  }
  if (tid == 0) {
    mbar_init(smem_u32(bar), 1);
    mbar_init(smem_u32(bar + 1), 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_base), 256);
  fence_proxy_async();
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t tmem = *tmem_base;
  const uint32_t lane_off = static_cast<uint32_t>(32 * (warp & 3)) << 16;
  const int rt = tid & 127;          // operand row of this thread within a tile
  const int part = tid >> 7;         // which column half it takes (PARTS = 2)
  // this thread's inter-stage twiddles W_N^(n2 k1): n2 = rt mod N2 is the
  // same for every tile and batch (128 is a multiple of N2), so they are
  // loaded once
  constexpr int KH = 32 / PARTS;
  float2 wtw[KH];
#pragma unroll
  for (int j = 0; j < KH; ++j) wtw[j] = __ldg(p.tc_tw + (rt % N2) * 32 + part * KH + j);
  const size_t total = static_cast<size_t>(p.nframes) * p.M * p.S;
  const size_t nbatch = (total + R - 1) / R;
  constexpr int bps = FC32 ? 8 : 4;
  static_assert(G::T1 == PARTS, "one stage-1 operand row per thread");
  static_assert(!FC32, "the tensor-core FFT takes sc16 rows");
  // sc16: this thread's stage-1 samples of the next batch are loaded while
  // the current batch runs (raw words, converted when the batch starts)
  const int b1 = (part * 128 + rt) / N2, n21 = (part * 128 + rt) % N2;
  uint32_t raw[32];
  auto load_raw = [&](size_t batch) {
    const size_t row = batch * R + b1;
    if (batch < nbatch && row < total) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(
          static_cast<const unsigned char*>(p.in) + (row * (N + p.cp) + p.cp) * bps);
#pragma unroll
      for (int n1 = 0; n1 < 32; ++n1) raw[n1] = __ldg(src + N2 * n1 + n21);
    } else {
#pragma unroll
      for (int n1 = 0; n1 < 32; ++n1) raw[n1] = 0x00000000u;   // converts to 0
    }
  };
  // MMA completion: stage 1 commits to bar[0], stage 2 to bar[1]; each has
  // at most one commit outstanding when it is waited on (a second commit to
  // one barrier before its wait would complete the next phase too, and the
  // parity wait could then not see the first)
  uint32_t phase[2] = {0, 0};
  bool timed_out = false;
  auto wait_mma = [&](int st) {
    if (!timed_out && !mbar_wait_bounded(smem_u32(bar + st), phase[st])) {
      timed_out = true;
      latch(p.status, kStTimeout);
    }
    phase[st] ^= 1;
    tmem_fence_after();
  };
  // operands of every thread visible to the MMA and this thread's TMEM
  // loads done before the issuing thread goes on
  auto to_mma = [&]() {
    fence_proxy_async();
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
  };
  // ---- stage-1 operands of a batch: row (b, n2) = x[N2 n1 + n2], n1 < 32,
  // from the raw words loaded ahead; then the next batch's words are loaded
  auto build_stage1 = [&](size_t batch) {
    float re[32], im[32];
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) {
      const float2 x = sc16_to_float2(raw[n1]);
      re[n1] = x.x;
      im[n1] = x.y;
    }
    store_row<32>(a1 + (2 * part) * G::A1_BYTES, a1 + (2 * part + 1) * G::A1_BYTES, rt, re, im,
                  split, bf16);
    load_raw(batch + gridDim.x);
  };
  auto issue_stage1 = [&]() {
    if (tid == 0) {
      for (int t = 0; t < G::T1; ++t)
        for (int term = 0; term < p.terms; ++term) {
          const uint32_t abase = smem_u32(a1 + (2 * t + (term == 2 ? 1 : 0)) * G::A1_BYTES);
          const uint32_t bbase = smem_u32(w1 + (term == 1 ? 1 : 0) * G::W1_BYTES);
          for (int kc = 0; kc < 4; ++kc)
            umma_f16(tmem + t * 64, tc_desc(abase + kc * 256, 64), tc_desc(bbase + kc * 256, 64),
                     umma_idesc(64, bf16), (term > 0 || kc > 0) ? 1u : 0u);
        }
      umma_commit(smem_u32(bar));
    }
  };
  auto issue_stage2 = [&]() {
    if (tid == 0) {
      for (int t = 0; t < G::T2; ++t)
        for (int term = 0; term < p.terms; ++term) {
          const uint32_t abase = smem_u32(a2 + (2 * t + (term == 2 ? 1 : 0)) * G::A2_BYTES);
          const uint32_t bbase = smem_u32(w2 + (term == 1 ? 1 : 0) * G::W2_BYTES);
          // A2 MN-major: 8-row groups 128 B apart, 8-column groups 2048 B
          // apart (16 row groups), two column groups per K = 16 step
          for (int kc = 0; kc < (2 * N2) / 16; ++kc)
            umma_f16(tmem + 128 + t * (2 * N2), umma_desc(abase + kc * 4096, 2048, 128),
                     tc_desc(bbase + kc * 256, 2 * N2), umma_idesc(2 * N2, bf16) | (1u << 15),
                     (term > 0 || kc > 0) ? 1u : 0u);
        }
      umma_commit(smem_u32(bar + 1));
    }
  };
  // Software pipeline over this block's batches: the stage-2 MMAs of batch
  // i run while the threads build the stage-1 operands of batch i + 1 (A1 is
  // free once batch i's stage-1 MMAs completed), and batch i + 1's stage-1
  // MMAs are queued behind them while batch i's output is stored.  The two
  // stages use separate TMEM columns, and every operand buffer is rewritten
  // only after the MMAs reading it have been waited for.
  if (blockIdx.x < nbatch) {
    load_raw(blockIdx.x);
    build_stage1(blockIdx.x);
    to_mma();
    issue_stage1();
  }
  for (size_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const size_t row0 = batch * R;
    const bool more = batch + gridDim.x < nbatch;
    wait_mma(0);   // stage 1 of this batch
    // ---- twiddle, scale by 2^-6 and store the stage-2 operand directly in
    // the MN-major layout: row m = (b, k1) of A2 is output k1 of batch row b,
    // column n2 (real) or N2 + n2 (imaginary) is this thread's D1 row, so a
    // thread holds one column of A2 for its k1 and writes 8 rows (16 bytes)
    // per store; with two threads per D1 row each takes 32 / PARTS of the k1
#pragma unroll
    for (int t = 0; t < G::T1; ++t) {
      float dr[KH], di[KH];
      Tmem<KH>::ld(tmem + lane_off + t * 64 + part * KH, dr);
      Tmem<KH>::ld(tmem + lane_off + t * 64 + 32 + part * KH, di);
      tmem_wait_ld();
      const int lr = t * 128 + rt;
      const int b = lr / N2, n2 = lr % N2;
#pragma unroll
      for (int j0 = 0; j0 < KH; j0 += 8) {
        uint32_t hr[4], lr_[4], hi_[4], li[4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          const float2 c0 = cmul(make_float2(dr[j0 + j], di[j0 + j]), wtw[j0 + j]);
          const float2 c1 = cmul(make_float2(dr[j0 + j + 1], di[j0 + j + 1]), wtw[j0 + j + 1]);
          const float r0 = c0.x * 0.015625f, r1 = c1.x * 0.015625f;
          const float i0 = c0.y * 0.015625f, i1 = c1.y * 0.015625f;
          if (bf16) {
            splitbf16x2(r0, r1, hr[j / 2], lr_[j / 2]);
            splitbf16x2(i0, i1, hi_[j / 2], li[j / 2]);
          } else {
            split16x2(r0, r1, hr[j / 2], lr_[j / 2]);
            split16x2(i0, i1, hi_[j / 2], li[j / 2]);
          }
        }
        const int m = b * 32 + part * KH + j0;           // first of 8 rows
        unsigned char* img = a2 + (2 * (m >> 7)) * G::A2_BYTES;
        const int ore = tc_mn_off(m & 127, n2);
        const int oim = tc_mn_off(m & 127, N2 + n2);
        *reinterpret_cast<uint4*>(img + ore) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
        *reinterpret_cast<uint4*>(img + oim) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
        if (split) {
          *reinterpret_cast<uint4*>(img + G::A2_BYTES + ore) = make_uint4(lr_[0], lr_[1], lr_[2], lr_[3]);
          *reinterpret_cast<uint4*>(img + G::A2_BYTES + oim) = make_uint4(li[0], li[1], li[2], li[3]);
        }
      }
    }
    to_mma();
    issue_stage2();
    if (more) {
      build_stage1(batch + gridDim.x);
      to_mma();
      issue_stage1();
    }
    wait_mma(1);   // stage 2 of this batch
    // ---- output: row (b, k1) holds X[k1 + 32 k2], re at column k2, im at N2 + k2
    const float so = p.inv_sqrtN * 64.f;
#pragma unroll
    for (int t = 0; t < G::T2; ++t) {
      const int lr = t * 128 + rt;
      const int b = lr / 32, k1 = lr % 32;
      const bool ok = row0 + b < total;
      float2* dst = p.Y_out + (row0 + b) * N + k1;
#pragma unroll
      for (int c0 = part * (N2 / PARTS); c0 < (part + 1) * (N2 / PARTS); c0 += 16) {
        float dr[16], di[16];
        Tmem<16>::ld(tmem + lane_off + 128 + t * (2 * N2) + c0, dr);
        Tmem<16>::ld(tmem + lane_off + 128 + t * (2 * N2) + N2 + c0, di);
        tmem_wait_ld();
        if (ok) {
#pragma unroll
          for (int j = 0; j < 16; ++j) dst[32 * (c0 + j)] = make_float2(dr[j] * so, di[j] * so);
        }
      }
    }
  }
  // every thread's last TMEM loads are done before the columns are freed
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

template <int LOG2N, bool FC32>
static cudaError_t launch_tc_t(const KParams& p, int grid, cudaStream_t st) {
  using G = TcGeo<LOG2N>;
  static int limit[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || limit[dev] < G::SMEM) {
    e = cudaFuncSetAttribute(tcfft_kernel<LOG2N, FC32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G::SMEM);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) limit[dev] = G::SMEM;
  }
  tcfft_kernel<LOG2N, FC32><<<grid, G::TT, G::SMEM, st>>>(p);
  return cudaGetLastError();
}

int tc_smem_bytes(int N) {
  switch (N) {
    case 512: return TcGeo<9>::SMEM;
    case 1024: return TcGeo<10>::SMEM;
    case 2048: return TcGeo<11>::SMEM;
  }
  return 0;
}

cudaError_t launch_tcfft(const KParams& p, int N, int grid, cudaStream_t st) {
  switch (N) {
    case 512: return launch_tc_t<9, false>(p, grid, st);
    case 1024: return launch_tc_t<10, false>(p, grid, st);
    case 2048: return launch_tc_t<11, false>(p, grid, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- staged receiver

constexpr int kYrxMaxThreads = 128;
constexpr int kYrxMaxD = 63;

// LS, MRC and demap from transformed symbols Y [F][M][S][N] (unitary): one
// thread per subcarrier k of one frame, the antenna loop in the thread (the
// MRC sum over antennas in a fixed order), packed bits through shared memory.
__global__ void __launch_bounds__(kYrxMaxThreads) yrx_kernel(const KParams p) {
  __shared__ uint8_t codes[kYrxMaxD * kYrxMaxThreads];
  const int N = p.N;
  const int T = blockDim.x;   // min(N, 128) subcarriers per block
  const int per = N / T;
  const int f = blockIdx.x / per;
  const int k0 = (blockIdx.x % per) * T;
  const int k = k0 + threadIdx.x;
  const float2 xs = p.xinv[k];                       // conj(X)/|X|^2/sqrt(N)
  const float sq = 1.0f / p.inv_sqrtN;
  const float2 xi = make_float2(xs.x * sq, xs.y * sq);   // conj(X)/|X|^2
  float2 P[kYrxMaxD];
  for (int d = 0; d < p.D; ++d) P[d] = make_float2(0.f, 0.f);
  float E = 0.f;
  for (int m = 0; m < p.M; ++m) {
    const float2* Ym = p.Y_out + (static_cast<size_t>(f) * p.M + m) * p.S * N;
    const float2 h = cmul(Ym[static_cast<size_t>(p.pilot_idx) * N + k], xi);
    p.H_out[(static_cast<size_t>(f) * p.M + m) * N + k] = h;
    E = fmaf(h.x, h.x, fmaf(h.y, h.y, E));
    for (int d = 0; d < p.D; ++d) {
      const int s = d < p.pilot_idx ? d : d + 1;
      const float2 y = Ym[static_cast<size_t>(s) * N + k];
      P[d].x = fmaf(h.x, y.x, fmaf(h.y, y.y, P[d].x));
      P[d].y = fmaf(h.x, y.y, fmaf(-h.y, y.x, P[d].y));
    }
  }
  const bool ok = (E > 0.f) && (E <= FLT_MAX);
  if (!ok) latch(p.status, kStDevice);
  const float ie = ok ? 1.0f / E : 0.f;
  for (int d = 0; d < p.D; ++d) {
    const float2 z = ok ? make_float2(P[d].x * ie, P[d].y * ie) : make_float2(0.f, 0.f);
    if (p.eq) p.eq[(static_cast<size_t>(f) * p.D + d) * N + k] = z;
    uint32_t code = gray(axis_level(z.x, p));
    if (p.axes == 2) code = (code << p.wbits) | gray(axis_level(z.y, p));
    codes[d * T + threadIdx.x] = static_cast<uint8_t>(code);
  }
  __syncthreads();
  const size_t frame_bytes = static_cast<size_t>(p.D) * N * p.q / 8;
  for (int it = threadIdx.x; it < p.D * (T / 8); it += T) {
    const int d = it / (T / 8);
    const int c8 = (it % (T / 8)) * 8;
    uint64_t acc = 0;
    for (int j = 0; j < 8; ++j) acc = (acc << p.q) | codes[d * T + c8 + j];
    uint8_t* dst = p.bits + f * frame_bytes + (static_cast<size_t>(d) * N + k0 + c8) * p.q / 8;
    for (int j = 0; j < p.q; ++j) dst[j] = static_cast<uint8_t>(acc >> (8 * (p.q - 1 - j)));
  }
}

cudaError_t launch_yrx(const KParams& p, int n_frames, cudaStream_t st) {
  const int T = p.N < kYrxMaxThreads ? p.N : kYrxMaxThreads;
  yrx_kernel<<<n_frames * (p.N / T), T, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace lsas
