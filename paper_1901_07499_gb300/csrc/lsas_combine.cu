// lsas_combine.cu -- combine step of the antenna-split receiver.
//
// Sec. IV proposes distributing the receiver when one server cannot take the
// data of every antenna.  MRC splits cleanly by antenna: each shard of
// antennas forms, per subcarrier, its partial sums sum conj(H) Y (every data
// symbol) and sum |H|^2 (frame_kernel in kModePartial).  This kernel adds the
// partials of G shards in shard order g = 0 .. G-1 (a fixed order, so the
// result does not depend on scheduling), forms z = P / E and finishes as the
// fused kernel does: Gray slicer, packed bits, optional z.
#include <cfloat>

#include <type_traits>

#include "lsas_kernels.cuh"

namespace lsas {

// small blocks: a single frame's 13 x 1024 / 8 threads spread over ~26 SMs
constexpr int kCombineThreads = 64;

// One thread per 8 consecutive points (data symbol d, subcarriers k0..k0+7)
// of one frame: it reads 64 B of partial sums and 32 B of energies per shard
// and writes the q bytes those 8 points pack into.  Partials are streamed
// (read once); energies are re-read once per data symbol and stay in cache.
__global__ void __launch_bounds__(kCombineThreads) combine_kernel(const KParams p) {
  const size_t per_frame = static_cast<size_t>(p.D) * p.N / 8;
  const size_t t = static_cast<size_t>(blockIdx.x) * kCombineThreads + threadIdx.x;
  if (t >= per_frame * static_cast<size_t>(p.nframes)) return;
  const int f = static_cast<int>(t / per_frame);
  const size_t r = t % per_frame;   // points 8r .. 8r+7 of the frame's d*N + k
  const int k0 = static_cast<int>((r * 8) % p.N);
  const size_t dn = static_cast<size_t>(p.D) * p.N;
  float2 P[8];
  float E[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    P[j] = make_float2(0.f, 0.f);
    E[j] = 0.f;
  }
  // unrolled so that several shards' loads are in flight at once (the sums
  // still run in shard order)
#pragma unroll 4
  for (int g = 0; g < p.shards; ++g) {
    const size_t gf = static_cast<size_t>(g) * p.nframes + f;
    const float4* Pg = reinterpret_cast<const float4*>(p.P_in + gf * dn + r * 8);
    const float4* Eg = reinterpret_cast<const float4*>(p.E_in + gf * p.N + k0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 v = __ldcs(Pg + j);
      P[2 * j].x += v.x;
      P[2 * j].y += v.y;
      P[2 * j + 1].x += v.z;
      P[2 * j + 1].y += v.w;
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float4 e = __ldg(Eg + j);
      E[4 * j] += e.x;
      E[4 * j + 1] += e.y;
      E[4 * j + 2] += e.z;
      E[4 * j + 3] += e.w;
    }
  }
  // one copy of the slicing per constellation, so that it has no branches
  auto codes_of = [&](auto tcount) {
    constexpr int T = decltype(tcount)::value;
    uint64_t a = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      // zero or non-finite energy: z = 0 and the frame is flagged
      const bool ok = (E[j] > 0.f) && (E[j] <= FLT_MAX);
      if (!ok) latch(p.status, kStDevice);
      const float ie = ok ? 1.0f / E[j] : 0.f;
      const float2 z = ok ? make_float2(P[j].x * ie, P[j].y * ie) : make_float2(0.f, 0.f);
      if (p.eq) p.eq[f * dn + r * 8 + j] = z;
      uint32_t code = gray(count_ge<T>(z.x, p.thr));
      if (p.axes == 2) code = (code << p.wbits) | gray(count_ge<T>(z.y, p.thr));
      a = (a << p.q) | code;
    }
    return a;
  };
  uint64_t acc;
  switch (p.nthr) {
    case 1: acc = codes_of(std::integral_constant<int, 1>{}); break;
    case 3: acc = codes_of(std::integral_constant<int, 3>{}); break;
    case 7: acc = codes_of(std::integral_constant<int, 7>{}); break;
    default: acc = codes_of(std::integral_constant<int, kMaxThresholds>{}); break;
  }
  uint8_t* dst = p.bits + f * (dn * p.q / 8) + r * p.q;
  for (int j = 0; j < p.q; ++j) dst[j] = static_cast<uint8_t>(acc >> (8 * (p.q - 1 - j)));
}

cudaError_t launch_combine(const KParams& p, cudaStream_t st) {
  const size_t n = static_cast<size_t>(p.nframes) * p.D * p.N / 8;
  const unsigned grid = static_cast<unsigned>((n + kCombineThreads - 1) / kCombineThreads);
  combine_kernel<<<grid, kCombineThreads, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace lsas
