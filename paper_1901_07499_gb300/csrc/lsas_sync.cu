// lsas_sync.cu -- packet detection and output reordering around the receiver.
//
// Sec. II-B: the received baseband is correlated with the maximum-length PN
// sequence that precedes each frame to find where the packet begins.  Here
// every antenna's capture is correlated with the PN chips and the powers are
// summed over antennas; the earliest lag of the largest sum is the preamble
// start, and the frame follows the preamble.  Sec. II-C: fftshift reorders
// the subcarriers so that the zero-frequency bin sits in the middle.
#include <type_traits>

#include "lsas_kernels.cuh"

namespace lsas {

constexpr int kPnThreads = 256;

// One block per frame.  For a chunk of kPnThreads lags at a time, every
// antenna row is staged through shared memory and each thread correlates its
// lag with the chips; then the block reduces (power, lag) to the largest
// power, the smallest lag on ties.
template <bool FC32>
__global__ void __launch_bounds__(kPnThreads) pn_kernel(const KParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  float2* tile = reinterpret_cast<float2*>(smem);
  float* pns = reinterpret_cast<float*>(tile + kPnThreads + p.pn_len);
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  const int span = kPnThreads + p.pn_len - 1;
  for (int i = tid; i < p.pn_len; i += kPnThreads) pns[i] = p.pn[i];
  float best = -1.f;
  int best_tau = 0;
  for (int tau0 = 0; tau0 < p.window; tau0 += kPnThreads) {
    float acc = 0.f;
    for (int m = 0; m < p.M; ++m) {
      __syncthreads();   // the previous tile is consumed
      const size_t row = (static_cast<size_t>(f) * p.M + m) * p.cap_len;
      for (int i = tid; i < span; i += kPnThreads) {
        const int idx = tau0 + i;
        float2 v = make_float2(0.f, 0.f);
        if (idx < p.cap_len) {
          if constexpr (FC32) v = __ldg(static_cast<const float2*>(p.in) + row + idx);
          else v = sc16_to_float2(__ldg(static_cast<const uint32_t*>(p.in) + row + idx));
        }
        tile[i] = v;
      }
      __syncthreads();
      float2 c = make_float2(0.f, 0.f);
      for (int n = 0; n < p.pn_len; ++n) {
        const float w = pns[n];
        c = __ffma2_rn(make_float2(w, w), tile[tid + n], c);
      }
      acc = fmaf(c.x, c.x, fmaf(c.y, c.y, acc));
    }
    const int tau = tau0 + tid;
    if (tau < p.window && acc > best) {   // lags grow: the earliest wins a tie
      best = acc;
      best_tau = tau;
    }
  }
  // block reduction of (power, lag)
  __shared__ float rv[kPnThreads / 32];
  __shared__ int rt[kPnThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int ot = __shfl_xor_sync(0xffffffffu, best_tau, o);
    if (ov > best || (ov == best && ot < best_tau)) {
      best = ov;
      best_tau = ot;
    }
  }
  if ((tid & 31) == 0) {
    rv[tid >> 5] = best;
    rt[tid >> 5] = best_tau;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < kPnThreads / 32; ++w)
      if (rv[w] > best || (rv[w] == best && rt[w] < best_tau)) {
        best = rv[w];
        best_tau = rt[w];
      }
    p.offsets[f] = best_tau;
    if (p.peaks) p.peaks[f] = best;
  }
}

// One block per (frame, antenna): copy the frame's S (N + CP) samples from
// offset + pn_len - backoff of the capture row into the contiguous frame
// layout.  A start outside the capture zero-fills the row and latches
// LSAS_ERR_DEVICE.
template <bool FC32>
__global__ void extract_kernel(const KParams p) {
  using W = typename std::conditional<FC32, uint2, uint32_t>::type;
  const int fm = blockIdx.x;
  const int f = fm / p.M;
  const int T = p.S * (p.N + p.cp);
  const long start = static_cast<long>(p.offsets_in[f]) + p.pn_len - p.backoff;
  W* dst = static_cast<W*>(const_cast<void*>(static_cast<const void*>(p.Y_out))) +
           static_cast<size_t>(fm) * T;
  if (start < 0 || start + T > p.cap_len) {
    if (threadIdx.x == 0) latch(p.status, kStDevice);
    for (int i = threadIdx.x; i < T; i += blockDim.x) dst[i] = W{};
    return;
  }
  const W* src = static_cast<const W*>(p.in) + static_cast<size_t>(fm) * p.cap_len + start;
  for (int i = threadIdx.x; i < T; i += blockDim.x) dst[i] = src[i];
}

// fftshift of complex rows of N (swap the halves of every row).
__global__ void shift_c64_kernel(float2* buf, size_t rows, int N) {
  const size_t half = static_cast<size_t>(N / 2);
  const size_t n = rows * half;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t r = i / half, k = i % half;
    float2* a = buf + r * N + k;
    const float2 t = a[0];
    a[0] = a[half];
    a[half] = t;
  }
}

// fftshift of packed bit rows (one data symbol = N q bits): swap the halves.
__global__ void shift_bytes_kernel(uint8_t* buf, size_t rows, int rowbytes) {
  const size_t half = static_cast<size_t>(rowbytes / 2);
  const size_t n = rows * half;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t r = i / half, k = i % half;
    uint8_t* a = buf + r * rowbytes + k;
    const uint8_t t = a[0];
    a[0] = a[half];
    a[half] = t;
  }
}

int pn_smem_bytes(int pn_len) { return (kPnThreads + pn_len) * 8 + pn_len * 4; }

cudaError_t launch_pn(const KParams& p, bool fc32, int n_frames, cudaStream_t st) {
  const int smem = pn_smem_bytes(p.pn_len);
  if (fc32) pn_kernel<true><<<n_frames, kPnThreads, smem, st>>>(p);
  else pn_kernel<false><<<n_frames, kPnThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_extract(const KParams& p, bool fc32, int n_frames, cudaStream_t st) {
  if (fc32) extract_kernel<true><<<n_frames * p.M, 256, 0, st>>>(p);
  else extract_kernel<false><<<n_frames * p.M, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_shift(void* buf, int kind, size_t rows, int N, int rowbytes, int sms,
                         cudaStream_t st) {
  const int grid = sms * 4;
  if (kind == 0) shift_c64_kernel<<<grid, 256, 0, st>>>(static_cast<float2*>(buf), rows, N);
  else shift_bytes_kernel<<<grid, 256, 0, st>>>(static_cast<uint8_t*>(buf), rows, rowbytes);
  return cudaGetLastError();
}

}  // namespace lsas
