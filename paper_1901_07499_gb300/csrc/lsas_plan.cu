// lsas_plan.cu -- host runtime and C ABI of liblsas (see include/lsas.h).
//
// A plan fixes one receiver configuration (M antennas, N subcarriers, CP,
// S symbols, pilot position, QAM order, input format) and owns the device
// tables its kernels read: the N-point twiddles W_N^i (computed here in
// double precision and rounded once), the LS pilot inverse
// conj(X)/|X|^2/sqrt(N) (Sec. II-C: LS is a division by the pilot), and a
// status word the kernels latch device-side conditions into.  Every argument
// is checked here before anything is enqueued.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lsas.h"
#include "lsas_kernels.cuh"
#include "lsas_hyb.cuh"
#include "lsas_pair.cuh"

namespace lsas {
cudaError_t launch_n64(int, bool, const KParams&, int, int, cudaStream_t);
cudaError_t launch_n128(int, bool, const KParams&, int, int, cudaStream_t);
cudaError_t launch_n256(int, bool, const KParams&, int, int, cudaStream_t);
cudaError_t launch_n512(int, bool, const KParams&, int, int, cudaStream_t);
cudaError_t launch_n1024(int, bool, const KParams&, int, int, cudaStream_t);
cudaError_t launch_n2048(int, bool, const KParams&, int, int, cudaStream_t);
cudaError_t launch_combine(const KParams&, cudaStream_t);
cudaError_t launch_tcfft(const KParams&, int N, int grid, cudaStream_t);
cudaError_t launch_yrx(const KParams&, int n_frames, cudaStream_t);
int tc_smem_bytes(int N);
cudaError_t dn_ls_tc(const KParams& k, const void* params_bf16, int n_frames, float* work,
                     float2* Hout, int* status, int sms, cudaStream_t st);
size_t dn_work_floats(int R, int N);
cudaError_t launch_pn(const KParams&, bool fc32, int n_frames, cudaStream_t);
cudaError_t launch_extract(const KParams&, bool fc32, int n_frames, cudaStream_t);
cudaError_t launch_shift(void* buf, int kind, size_t rows, int N, int rowbytes, int sms,
                         cudaStream_t);
int pn_smem_bytes(int pn_len);
bool tc_tables(int N, std::vector<uint16_t>& w1, std::vector<uint16_t>& w2,
               std::vector<float2>& tw);
}  // namespace lsas

using namespace lsas;

namespace {

constexpr int kSmemLimit = 232448;   // opt-in dynamic shared memory per block
constexpr size_t kTailBytes = 96u << 20;   // cap of a plan's split-tail partial sums
// Share of a fused block's time that does not shrink with its antenna count
// (the group-end reductions, demap and pack), for the split decision, from
// single-frame timings on GB300: about 0.08 for the per-warp kernel
// (N <= 1024, 64 antennas) and 0.035 for the warp-pair kernel (N = 2048,
// 128 antennas), whose group ends weigh less against its longer steps.
constexpr double kBlockFixedWarp = 0.08;
constexpr double kBlockFixedPair = 0.035;
constexpr int kHostChunk = 64;       // frames per transfer chunk (host path)
constexpr int kMaxPnLen = 1024;      // longest PN sequence lsas_plan_set_pn takes

struct Geometry {
  int A, L, T;
  int Af;   // antennas per step of the fused kernel (frame launches)
  int nslots, groups, dg, smem_frame;
  int smem_est, smem_fft, fft_slots;
  int tmem_cols, tmem_cth;
  int hybrid;   // N = 1024, sc16: fused calls with aligned rows use hyb_kernel
};

}  // namespace

struct lsas_plan_s {
  int M, N, cp, S, pilot_idx, Q, q, D;
  int wbits, axes, nthr;
  float thr[kMaxThresholds];
  lsas_input_fmt fmt;
  int max_frames;
  int device;
  float2* d_twP = nullptr;
  float2* d_xinv = nullptr;
  int* d_status = nullptr;
  float2 w32[16], w32n[16];
  // tensor-core FFT tables (N = 512 .. 2048)
  void* d_tc_w1 = nullptr;
  void* d_tc_w2 = nullptr;
  float2* d_tc_tw = nullptr;
  int sms = 0;
  // packet detection: PN chips (lsas_plan_set_pn)
  float* d_pn = nullptr;
  int pn_len = 0;
  int fault = 0;   // test hook of the bounded waits (lsas_plan_set_fault)
  bool allow_hybrid = false;   // LSAS_FUSED_KERNEL = "tensor" at creation
  bool twin = true;            // sc16: two symbols per step where it pays (LSAS_FUSED_KERNEL)
  void* d_split_scratch = nullptr;   // device address of g_split_scratch on this device
  // lsas_run_frame: the frames after a batch's last whole wave of blocks (all
  // of them, for a batch smaller than one wave) may run split into equal
  // antenna shards so that they fill the GPU; their partial sums live here,
  // P [G][frames][D][N] complex then E [G][frames][N]
  float* d_tail = nullptr;
  int tail_units = 0;               // shard-frames d_tail holds
  int batch_split = 1;              // lsas_plan_set_batch_split: 0 off, 1 per batch, 2 fixed
  cudaEvent_t tail_ev = nullptr;    // the last split's combine has read d_tail
  std::mutex tail_mu;
  size_t dev_bytes = 0;             // device memory allocated at creation
  Geometry geo;
  LaunchFn launch = nullptr;
  // host-transfer staging (lsas_run_frame_host), allocated on first use
  void* d_in_stage[2] = {nullptr, nullptr};
  float2* d_H_stage[2] = {nullptr, nullptr};
  uint8_t* d_bits_stage[2] = {nullptr, nullptr};
  float2* d_eq_stage[2] = {nullptr, nullptr};
  cudaStream_t up_stream = nullptr, down_stream = nullptr;
  cudaEvent_t ev_up[2] = {nullptr, nullptr};
  cudaEvent_t ev_k[2] = {nullptr, nullptr};
  cudaEvent_t ev_down[2] = {nullptr, nullptr};
  // call timing (LSAS_PROFILE=1 at creation, or lsas_plan_set_profile)
  struct ProfRec {
    const char* name;
    cudaEvent_t a, b;   // null for a call timed on the host clock
    double host_ms;
  };
  bool prof = false;
  std::mutex prof_mu;
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  std::map<std::string, std::pair<uint64_t, double>> prof_acc;
};

namespace {

cudaEvent_t prof_event(lsas_plan p) {   // caller holds prof_mu
  if (!p->prof_pool.empty()) {
    cudaEvent_t e = p->prof_pool.back();
    p->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Times one library call while the plan's profiling is on: events on the
// call's stream around what it enqueues, or the host clock for a call that
// synchronises before it returns.  Records are folded by lsas_plan_profile.
class ProfScope {
 public:
  ProfScope(lsas_plan p, const char* name, void* stream, bool host = false)
      : p_(p && p->prof ? p : nullptr), name_(name), st_(static_cast<cudaStream_t>(stream)),
        host_(host) {
    if (!p_) return;
    if (host_) {
      t0_ = std::chrono::steady_clock::now();
      return;
    }
    std::lock_guard<std::mutex> lock(p_->prof_mu);
    a_ = prof_event(p_);
    if (a_ && cudaEventRecord(a_, st_) != cudaSuccess) {
      cudaGetLastError();
      p_->prof_pool.push_back(a_);
      a_ = nullptr;
    }
  }
  ~ProfScope() {
    if (!p_) return;
    std::lock_guard<std::mutex> lock(p_->prof_mu);
    if (host_) {
      const double ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0_).count();
      p_->prof_recs.push_back({name_, nullptr, nullptr, ms});
      return;
    }
    if (!a_) return;
    cudaEvent_t b = prof_event(p_);
    if (b && cudaEventRecord(b, st_) == cudaSuccess) {
      p_->prof_recs.push_back({name_, a_, b, 0.0});
    } else {
      cudaGetLastError();
      p_->prof_pool.push_back(a_);
      if (b) p_->prof_pool.push_back(b);
    }
  }
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  lsas_plan p_;
  const char* name_;
  cudaStream_t st_;
  bool host_;
  cudaEvent_t a_ = nullptr;
  std::chrono::steady_clock::time_point t0_;
};

}  // namespace

namespace {

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2i(int x) {
  int r = 0;
  while ((1 << r) < x) ++r;
  return r;
}

size_t in_bytes_per_frame(int M, int N, int cp, int S, lsas_input_fmt fmt) {
  return static_cast<size_t>(M) * S * (N + cp) * (fmt == LSAS_IN_SC16 ? 4 : 8);
}
// Whether lsas_run_frame_host copies only the samples after each cyclic
// prefix (rows of at least 1 KB kept).
bool host_strips_cp(int N, int cp, lsas_input_fmt fmt) {
  return cp > 0 && static_cast<size_t>(N) * (fmt == LSAS_IN_SC16 ? 4 : 8) >= 1024;
}
size_t bits_bytes_per_frame(int N, int S, int Q) {
  return static_cast<size_t>(S - 1) * N * ilog2i(Q) / 8;
}

LaunchFn launcher_for(int N) {
  switch (N) {
    case 64: return launch_n64;
    case 128: return launch_n128;
    case 256: return launch_n256;
    case 512: return launch_n512;
    case 1024: return launch_n1024;
    case 2048: return launch_n2048;
    default: return nullptr;
  }
}

// Choose the staging depth (slots) and the data symbols per group so that the
// fused kernel fits the shared memory of one SM, its accumulators fit tensor
// memory, and the demapped codes fit the staging ring they reuse: prefer one
// data-symbol group (no second pass over H), then the deepest ring.
bool plan_geometry(int M, int N, int D, lsas_input_fmt fmt, bool allow_hybrid, Geometry* g) {
  g->A = geo_A(N);
  g->Af = geo_A(N);
  g->L = N / 32;
  g->T = geo_T(N);
  const int bps = fmt == LSAS_IN_SC16 ? 4 : 8;
  (void)M;
  const int own = geo_OWN(N);
  const int dg_tmem = (512 - own) / (2 * own);
  bool found = false;
  for (int groups = (D + dg_tmem - 1) / dg_tmem; groups <= D && !found; ++groups) {
    const int dg = (D + groups - 1) / groups;
    for (int slots = kMaxSlots; slots >= 2; --slots) {
      const Layout l = make_layout(N, bps, slots, 2);
      if (l.total > kSmemLimit || dg * N > slots * geo_A(N) * l.team_stage) continue;
      g->groups = groups;
      g->dg = dg;
      g->nslots = slots;
      g->smem_frame = l.total;
      found = true;
      break;
    }
  }
  if (!found) return false;
  g->tmem_cols = tmem_alloc_cols(N, g->dg);
  g->tmem_cth = tmem_cols_thread(N, g->dg);
  if (N <= 1024) {
    // per-warp kernel: TMEM bounds the data symbols per group; the deepest
    // staging ring that fits (at most three rows per warp for N = 1024,
    // which measured faster there than four), with room for one symbol of
    // every warp's partial sums in the per-warp regions
    found = false;
    const int dgmax = wgeo_dg_max(N, bps);
    const int max_slots = N == 1024 ? 3 : kMaxSlots;
    for (int groups = (D + dgmax - 1) / dgmax; groups <= D && !found; ++groups) {
      const int dg = (D + groups - 1) / groups;
      for (int slots = max_slots; slots >= 2; --slots) {
        const WLayout l = make_wlayout(N, bps, slots, dg);
        if (l.total > kSmemLimit || l.warp_bytes < N * 8) continue;
        g->groups = groups;
        g->dg = dg;
        g->nslots = slots;
        g->smem_frame = l.total;
        g->T = 32 * wgeo_warps(bps);
        g->Af = wgeo_A(N);
        g->tmem_cols = kWTmemCols;
        g->tmem_cth = wgeo_tmem_warp(wgeo_warps(bps));
        found = true;
        break;
      }
    }
    if (!found) return false;
  } else if (fmt == LSAS_IN_SC16) {
    // N = 2048 from sc16 rows: pipelines of warp pairs, the same bounds
    // (TMEM per warp, the deepest ring that fits)
    found = false;
    const int dgmax = pgeo_dg_max();
    for (int groups = (D + dgmax - 1) / dgmax; groups <= D && !found; ++groups) {
      const int dg = (D + groups - 1) / groups;
      for (int slots = kMaxSlots; slots >= 2; --slots) {
        const PLayout l = make_playout(slots, dg);
        if (l.total > kSmemLimit || l.pair_bytes < N * 8) continue;
        g->groups = groups;
        g->dg = dg;
        g->nslots = slots;
        g->smem_frame = l.total;
        g->T = kPThreads;
        g->Af = 1;
        g->tmem_cols = kWTmemCols;
        g->tmem_cth = kPTmemWarp;
        found = true;
        break;
      }
    }
    if (!found) return false;
  }
  g->hybrid = 0;
  if (allow_hybrid && N == 1024 && fmt == LSAS_IN_SC16) {
    // the tensor-core kernel's TMEM holds two data symbols per warp; the
    // per-warp kernel (unaligned rows) then runs the same groups
    const int groups = (D + kHyDgMax - 1) / kHyDgMax;
    const int dg = (D + groups - 1) / groups;
    const WLayout l = make_wlayout(N, bps, g->nslots, dg);
    if (l.total <= kSmemLimit) {
      g->groups = groups;
      g->dg = dg;
      g->smem_frame = l.total;
      g->hybrid = 1;
    }
  }
  g->smem_est = make_layout(N, bps, 1, 1).total;
  g->fft_slots = 2;
  g->smem_fft = make_layout(N, bps, 2, 1).total;
  return true;
}

// W_32^e = exp(-2j pi e / 32) as {Re, Im} and {-Im, Re}, e < 16.
void fill_w32(float2* w, float2* wn) {
  for (int e = 0; e < 16; ++e) {
    const double a = -2.0 * M_PI * e / 32.0;
    const float c = static_cast<float>(std::cos(a)), s = static_cast<float>(std::sin(a));
    w[e] = make_float2(c, s);
    wn[e] = make_float2(-s, c);
  }
}

// W_N^e = exp(-2j pi e / N), computed in double precision and rounded once.
float2 tw2(long e, int N) {
  const double a = -2.0 * M_PI * static_cast<double>(e % N) / N;
  return make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
}

// Twiddles of the FFT passes after the first, in the order the kernels read
// them (see pass_tw_count in lsas_kernels.cuh).
std::vector<float2> pass_twiddles(int N) {
  std::vector<float2> t(pass_tw_count(N));
  if (N <= 1024) {
    const int R2 = N / 32;
    for (int r = 0; r < R2; ++r)
      for (int j = 0; j < 32; ++j) t[r * 32 + j] = tw2(static_cast<long>(j) * r, N);
  } else {
    for (int r = 0; r < 8; ++r)
      for (int j = 0; j < 32; ++j) t[r * 32 + j] = tw2(8L * j * r, N);
    for (int r = 0; r < 8; ++r)
      for (int j = 0; j < 256; ++j) t[256 + r * 256 + j] = tw2(static_cast<long>(j) * r, N);
  }
  return t;
}

lsas_status upload_pilot(lsas_plan p, const double* re, const double* im) {
  std::vector<float2> xi(p->N);
  const double s = 1.0 / std::sqrt(static_cast<double>(p->N));
  for (int k = 0; k < p->N; ++k) {
    const double m2 = re[k] * re[k] + im[k] * im[k];
    if (!(m2 > 0.0) || !std::isfinite(m2)) return LSAS_ERR_INVALID_ARG;
    xi[k] = make_float2(static_cast<float>(re[k] / m2 * s), static_cast<float>(-im[k] / m2 * s));
  }
  if (cudaMemcpy(p->d_xinv, xi.data(), sizeof(float2) * p->N, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

bool aligned16(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

void base_params(lsas_plan p, KParams* k) {
  std::memset(k, 0, sizeof(*k));
  k->twP = p->d_twP;
  k->xinv = p->d_xinv;
  k->status = p->d_status;
  k->fault = p->fault;
  k->hybrid = p->geo.hybrid;
  // two symbols per step: N = 1024 and 2048 always; N = 512 and 256 only
  // with enough antennas (each lane keeps 32 subcarriers of its antenna, so
  // the data symbols take four groups where the one-symbol kernel needs one
  // at N = 256).  Decided per plan on its total antenna count, so that the
  // antenna shards of a split batch run the same arithmetic as a whole frame.
  k->twin = (p->twin && p->fmt == LSAS_IN_SC16 &&
             (p->N >= 1024 || (p->N == 512 && p->M >= 32) || (p->N == 256 && p->M >= 128)))
                ? 1 : 0;
  k->tc_w1 = p->d_tc_w1;
  k->M = p->M;
  k->m0 = 0;
  k->Mtot = p->M;
  k->N = p->N;
  k->S = p->S;
  k->cp = p->cp;
  k->pilot_idx = p->pilot_idx;
  k->D = p->D;
  k->chunks = (p->M + p->geo.A - 1) / p->geo.A;
  k->groups = p->geo.groups;
  k->dg = p->geo.dg;
  k->nslots = p->geo.nslots;
  k->tmem_cols = p->geo.tmem_cols;
  k->tmem_cth = p->geo.tmem_cth;
  k->q = p->q;
  k->wbits = p->wbits;
  k->axes = p->axes;
  k->nthr = p->nthr;
  k->inv_sqrtN = static_cast<float>(1.0 / std::sqrt(static_cast<double>(p->N)));
  for (int i = 0; i < kMaxThresholds; ++i) k->thr[i] = p->thr[i];
  for (int i = 0; i < 16; ++i) {
    k->w32[i] = p->w32[i];
    k->w32n[i] = p->w32n[i];
  }
}

// Bulk copies need 16-byte aligned rows: every row start
// ((f M + m) S + s)(N + CP) + CP samples from a 16-byte aligned base.
bool tma_ok(lsas_plan p, const void* d_in) {
  const int bps = p->fmt == LSAS_IN_SC16 ? 4 : 8;
  return aligned16(d_in) && ((p->N + p->cp) * bps) % 16 == 0 && (p->cp * bps) % 16 == 0;
}

lsas_status set_device(lsas_plan p) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return LSAS_ERR_CUDA;
  if (cur != p->device && cudaSetDevice(p->device) != cudaSuccess) return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status check_frames(lsas_plan p, int n_frames) {
  if (n_frames < 0) return LSAS_ERR_INVALID_ARG;
  if (n_frames > p->max_frames) return LSAS_ERR_CAPACITY;
  return LSAS_OK;
}

lsas_status launch_frame(lsas_plan p, const void* d_in, int n_frames, float* d_H,
                         const float* d_Hin, uint8_t* d_bits, float* d_eq, int mode,
                         cudaStream_t st) {
  KParams k;
  base_params(p, &k);
  k.in = d_in;
  k.H_out = reinterpret_cast<float2*>(d_H);
  k.H_in = reinterpret_cast<const float2*>(d_Hin);
  k.bits = d_bits;
  k.eq = reinterpret_cast<float2*>(d_eq);
  k.mode = mode;
  k.chunks = (p->M + p->geo.Af - 1) / p->geo.Af;
  k.use_tma = tma_ok(p, d_in) ? 1 : 0;
  if (p->launch(kKindFrame, p->fmt == LSAS_IN_FC32, k, n_frames, p->geo.smem_frame, st) !=
      cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

// Antenna shards G for nf frames that do not fill a whole wave of blocks
// (one block per SM): the split runs nf * G blocks of M / G antennas each,
// ceil(nf G / sms) waves of about (1 - f) / G + f of a frame's block time
// (f: kBlockFixedWarp or kBlockFixedPair), against one wave unsplit.  Equal
// shards only (one launch), each with at least one antenna per pipeline of
// the fused kernel, nf G within cap; 1 when no split saves 10 % of the wave.
int best_shards(lsas_plan p, int nf, long cap) {
  const int pipes = p->N <= 1024 ? wgeo_warps(p->fmt == LSAS_IN_SC16 ? 4 : 8)
                                  : (p->fmt == LSAS_IN_SC16 ? kPPairs : 1);
  const int min_ant = pipes * p->geo.Af;
  const double fixed = p->N > 1024 ? kBlockFixedPair : kBlockFixedWarp;
  double best = 0.9;
  int bestG = 1;
  for (int G = 2; G <= 32; G *= 2) {
    if (p->M % G != 0 || p->M / G < min_ant) continue;
    if (static_cast<long>(nf) * G > cap) continue;
    const double waves = std::ceil(static_cast<double>(nf) * G / p->sms);
    const double t = waves * ((1.0 - fixed) / G + fixed);
    if (t < best) {
      best = t;
      bestG = G;
    }
  }
  return bestG;
}

int tail_shards(lsas_plan p, int nf) {
  if (nf <= 0 || p->batch_split == 0 || p->tail_units == 0 || p->geo.hybrid) return 1;
  if (p->batch_split == 2) {
    // one shard count for every batch: the single frame's choice, among the
    // counts whose scratch holds a batch of max_frames
    return best_shards(p, 1, p->tail_units / (p->max_frames > 0 ? p->max_frames : 1));
  }
  return best_shards(p, nf, p->tail_units);
}

// Frames [f0, f0 + nf) of a lsas_run_frame batch as G antenna shards: the
// fused kernel's partial mode writes the shards' partial sums and H, the
// combine kernel forms z and the bits.  Calls on different streams share
// d_tail: each waits for the previous split's combine.
lsas_status run_split_tail(lsas_plan p, const void* d_in, int f0, int nf, int G, float* d_H,
                           uint8_t* d_bits, float* d_eq, cudaStream_t st) {
  const size_t in_b = in_bytes_per_frame(p->M, p->N, p->cp, p->S, p->fmt);
  const size_t bits_b = bits_bytes_per_frame(p->N, p->S, p->Q);
  const unsigned char* in = static_cast<const unsigned char*>(d_in) + f0 * in_b;
  float* P = p->d_tail;
  float* E = P + static_cast<size_t>(G) * nf * p->D * p->N * 2;
  std::lock_guard<std::mutex> lock(p->tail_mu);
  if (cudaStreamWaitEvent(st, p->tail_ev, 0) != cudaSuccess) return LSAS_ERR_CUDA;
  KParams k;
  base_params(p, &k);
  k.in = in;
  k.H_out = reinterpret_cast<float2*>(d_H + static_cast<size_t>(f0) * p->M * p->N * 2);
  k.P_out = reinterpret_cast<float2*>(P);
  k.E_out = E;
  k.M = p->M / G;
  k.shard_y = k.M;
  k.grid_y = G;
  // small batches: one block per data-symbol group as well (each repeats
  // the pilot transform), so a frame's groups also run side by side, as in
  // the one-launch static split
  k.group_z = ((p->N <= 1024 || p->fmt == LSAS_IN_SC16) && p->geo.groups > 1 &&
               nf * G * 2 <= p->sms) ? 1 : 0;
  k.chunks = (k.M + p->geo.Af - 1) / p->geo.Af;
  k.mode = kModePartial;
  k.use_tma = tma_ok(p, in) ? 1 : 0;
  lsas_status s = LSAS_OK;
  if (p->launch(kKindFrame, p->fmt == LSAS_IN_FC32, k, nf, p->geo.smem_frame, st) != cudaSuccess) {
    s = LSAS_ERR_CUDA;
  } else {
    KParams c;
    base_params(p, &c);
    c.P_in = reinterpret_cast<const float2*>(P);
    c.E_in = E;
    c.shards = G;
    c.nframes = nf;
    c.bits = d_bits + f0 * bits_b;
    c.eq = d_eq ? reinterpret_cast<float2*>(d_eq + static_cast<size_t>(f0) * p->D * p->N * 2)
                : nullptr;
    if (launch_combine(c, st) != cudaSuccess) s = LSAS_ERR_CUDA;
  }
  if (cudaEventRecord(p->tail_ev, st) != cudaSuccess) s = LSAS_ERR_CUDA;
  return s;
}

}  // namespace

// ---------------------------------------------------------------------------
// Fixed device scratch for lsas_run_frame_split_static: the antenna-split
// partial sums of one call live here instead of in caller or library
// allocations, so that the call allocates nothing.  One array per device
// (a __device__ variable exists once in every context).  Host code cannot
// use the symbol's name as a device address: lsas_plan_create looks the
// address up with cudaGetSymbolAddress, with the plan's device current, and
// keeps it in the plan, so that loading the module and committing the array
// happen there and never inside the entry point.  Calls that overlap in time
// on one device share the array and race.
static __device__ __align__(256) unsigned char g_split_scratch[LSAS_STATIC_SCRATCH_BYTES];

extern "C" {

const char* lsas_status_str(lsas_status s) {
  switch (s) {
    case LSAS_OK: return "LSAS_OK";
    case LSAS_ERR_INVALID_ARG: return "LSAS_ERR_INVALID_ARG";
    case LSAS_ERR_UNSUPPORTED: return "LSAS_ERR_UNSUPPORTED";
    case LSAS_ERR_OOM: return "LSAS_ERR_OOM";
    case LSAS_ERR_CAPACITY: return "LSAS_ERR_CAPACITY";
    case LSAS_ERR_CUDA: return "LSAS_ERR_CUDA";
    case LSAS_ERR_TIMEOUT: return "LSAS_ERR_TIMEOUT";
    case LSAS_ERR_DEVICE: return "LSAS_ERR_DEVICE";
  }
  return "LSAS_ERR_UNKNOWN";
}

lsas_status lsas_check_config(int M, int N, int cp_len, int n_sym, int pilot_idx,
                              int qam_order) {
  if (M < 1 || M > 256) return LSAS_ERR_INVALID_ARG;
  if (!is_pow2(N) || N < 64 || N > 2048) return LSAS_ERR_INVALID_ARG;
  if (cp_len < 0 || cp_len >= N) return LSAS_ERR_INVALID_ARG;
  if (n_sym < 2 || n_sym > 64) return LSAS_ERR_INVALID_ARG;
  if (pilot_idx < 0 || pilot_idx >= n_sym) return LSAS_ERR_INVALID_ARG;
  if (qam_order != 2 && qam_order != 4 && qam_order != 16 && qam_order != 64 &&
      qam_order != 256)
    return LSAS_ERR_INVALID_ARG;
  return LSAS_OK;
}

lsas_status lsas_frame_bytes(int M, int N, int cp_len, int n_sym, int qam_order,
                             lsas_input_fmt fmt, size_t out[4]) {
  if (!out) return LSAS_ERR_INVALID_ARG;
  lsas_status s = lsas_check_config(M, N, cp_len, n_sym, 0, qam_order);
  if (s != LSAS_OK) return s;
  if (fmt != LSAS_IN_SC16 && fmt != LSAS_IN_FC32) return LSAS_ERR_INVALID_ARG;
  out[0] = in_bytes_per_frame(M, N, cp_len, n_sym, fmt);
  out[1] = static_cast<size_t>(M) * N * 8;
  out[2] = bits_bytes_per_frame(N, n_sym, qam_order);
  out[3] = static_cast<size_t>(n_sym - 1) * N * 8;
  return LSAS_OK;
}

lsas_status lsas_plan_create(int M, int N, int cp_len, int n_sym, int pilot_idx,
                             int qam_order, lsas_plan* out) {
  if (!out) return LSAS_ERR_INVALID_ARG;
  *out = nullptr;
  lsas_status s = lsas_check_config(M, N, cp_len, n_sym, pilot_idx, qam_order);
  if (s != LSAS_OK) return s;
  lsas_plan p = new (std::nothrow) lsas_plan_s();
  if (!p) return LSAS_ERR_OOM;
  p->M = M;
  p->N = N;
  p->cp = cp_len;
  p->S = n_sym;
  p->pilot_idx = pilot_idx;
  p->Q = qam_order;
  p->q = ilog2i(qam_order);
  p->D = n_sym - 1;
  p->fmt = LSAS_IN_SC16;
  p->max_frames = 1024;
  // per-axis decision boundaries (2b - L) A of unit-energy Gray QAM
  int L;
  double A;
  if (qam_order == 2) {
    L = 2;
    A = 1.0;
    p->axes = 1;
    p->wbits = 1;
  } else {
    L = static_cast<int>(std::lround(std::sqrt(static_cast<double>(qam_order))));
    A = 1.0 / std::sqrt(2.0 * (qam_order - 1) / 3.0);
    p->axes = 2;
    p->wbits = ilog2i(L);
  }
  p->nthr = L - 1;
  for (int b = 0; b < kMaxThresholds; ++b)
    p->thr[b] = b < L - 1 ? static_cast<float>((2.0 * (b + 1) - L) * A) : 0.f;
  fill_w32(p->w32, p->w32n);
  p->launch = launcher_for(N);
  {
    const char* e = std::getenv("LSAS_PROFILE");
    p->prof = e && e[0] == '1';
  }
  {
    // Fused kernel from sc16 rows: by default two symbols per step where it
    // pays (twin_kernel, twinpair_kernel); LSAS_FUSED_KERNEL=warp selects one
    // symbol per step (warp_kernel, pair_kernel) and LSAS_FUSED_KERNEL=tensor
    // at N = 1024 the second FFT pass on the tensor cores (hyb_kernel), both
    // measured slower
    const char* e = std::getenv("LSAS_FUSED_KERNEL");
    p->allow_hybrid = e && std::strcmp(e, "tensor") == 0;
    p->twin = !(e && (std::strcmp(e, "warp") == 0 || std::strcmp(e, "tensor") == 0));
  }
  if (!plan_geometry(M, N, p->D, p->fmt, p->allow_hybrid, &p->geo)) {
    delete p;
    return LSAS_ERR_UNSUPPORTED;
  }
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return LSAS_ERR_CUDA;
  }
  const std::vector<float2> tw = pass_twiddles(N);
  if (cudaMalloc(&p->d_twP, sizeof(float2) * tw.size()) != cudaSuccess ||
      cudaMalloc(&p->d_xinv, sizeof(float2) * N) != cudaSuccess ||
      cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    lsas_plan_destroy(p);
    return LSAS_ERR_OOM;
  }
  p->dev_bytes = sizeof(float2) * (tw.size() + N) + sizeof(int);
  std::vector<uint16_t> tcw1, tcw2;
  std::vector<float2> tctw;
  if (tc_tables(N, tcw1, tcw2, tctw)) {
    if (cudaMalloc(&p->d_tc_w1, tcw1.size() * 2) != cudaSuccess ||
        cudaMalloc(&p->d_tc_w2, tcw2.size() * 2) != cudaSuccess ||
        cudaMalloc(&p->d_tc_tw, tctw.size() * sizeof(float2)) != cudaSuccess) {
      cudaGetLastError();
      lsas_plan_destroy(p);
      return LSAS_ERR_OOM;
    }
    p->dev_bytes += (tcw1.size() + tcw2.size()) * 2 + tctw.size() * sizeof(float2);
    if (cudaMemcpy(p->d_tc_w1, tcw1.data(), tcw1.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_tc_w2, tcw2.data(), tcw2.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_tc_tw, tctw.data(), tctw.size() * sizeof(float2), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      lsas_plan_destroy(p);
      return LSAS_ERR_CUDA;
    }
  }
  if (cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    lsas_plan_destroy(p);
    return LSAS_ERR_CUDA;
  }
  {
    // partial sums of split tails (lsas_run_frame): up to three waves of
    // shard-frames, within kTailBytes; without them every batch runs unsplit
    const size_t unit = (static_cast<size_t>(p->D) * N * 2 + N) * sizeof(float);
    const size_t units = std::min(static_cast<size_t>(3 * p->sms), kTailBytes / unit);
    if (units >= 2 && cudaMalloc(&p->d_tail, units * unit) == cudaSuccess &&
        cudaEventCreateWithFlags(&p->tail_ev, cudaEventDisableTiming) == cudaSuccess) {
      p->tail_units = static_cast<int>(units);
      p->dev_bytes += units * unit;
    } else {
      cudaGetLastError();
      cudaFree(p->d_tail);
      p->d_tail = nullptr;
      p->tail_units = 0;
    }
  }
  // address of the static split scratch on this device (the device is
  // current here); lsas_run_frame_split_static never looks it up itself
  if (cudaGetSymbolAddress(&p->d_split_scratch, g_split_scratch) != cudaSuccess) {
    cudaGetLastError();
    lsas_plan_destroy(p);
    return LSAS_ERR_CUDA;
  }
  std::vector<double> one(N, 1.0), zero(N, 0.0);
  if (cudaMemcpy(p->d_twP, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess ||
      upload_pilot(p, one.data(), zero.data()) != LSAS_OK) {
    lsas_plan_destroy(p);
    return LSAS_ERR_CUDA;
  }
  *out = p;
  return LSAS_OK;
}

lsas_status lsas_plan_set(lsas_plan p, lsas_input_fmt fmt, int max_frames) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  if (fmt != LSAS_IN_SC16 && fmt != LSAS_IN_FC32) return LSAS_ERR_INVALID_ARG;
  if (max_frames < 1) return LSAS_ERR_INVALID_ARG;
  Geometry g;
  if (!plan_geometry(p->M, p->N, p->D, fmt, p->allow_hybrid, &g)) return LSAS_ERR_UNSUPPORTED;
  const bool realloc = fmt != p->fmt || max_frames != p->max_frames;
  p->fmt = fmt;
  p->max_frames = max_frames;
  p->geo = g;
  if (realloc) {
    // host-transfer staging depends on both; drop it, the next host call
    // allocates it again
    if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
    cudaDeviceSynchronize();
    for (int i = 0; i < 2; ++i) {
      cudaFree(p->d_in_stage[i]);
      cudaFree(p->d_H_stage[i]);
      cudaFree(p->d_bits_stage[i]);
      cudaFree(p->d_eq_stage[i]);
      p->d_in_stage[i] = nullptr;
      p->d_H_stage[i] = nullptr;
      p->d_bits_stage[i] = nullptr;
      p->d_eq_stage[i] = nullptr;
    }
  }
  return LSAS_OK;
}

lsas_status lsas_plan_set_pilot(lsas_plan p, const float* host_pilot_iq) {
  if (!p || !host_pilot_iq) return LSAS_ERR_INVALID_ARG;
  std::vector<double> re(p->N), im(p->N);
  for (int k = 0; k < p->N; ++k) {
    re[k] = host_pilot_iq[2 * k];
    im[k] = host_pilot_iq[2 * k + 1];
  }
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  return upload_pilot(p, re.data(), im.data());
}

lsas_status lsas_fft(lsas_plan p, const void* d_in, int n_frames, float* d_Y, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (n_frames == 0) return LSAS_OK;
  if (!d_in || !d_Y) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  KParams k;
  base_params(p, &k);
  k.in = d_in;
  k.Y_out = reinterpret_cast<float2*>(d_Y);
  k.nslots = p->geo.fft_slots;
  k.use_tma = tma_ok(p, d_in) ? 1 : 0;
  const int grid = n_frames * k.chunks;
  ProfScope prof(p, "lsas_fft", stream);
  if (p->launch(kKindFft, p->fmt == LSAS_IN_FC32, k, grid, p->geo.smem_fft,
                static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status lsas_estimate(lsas_plan p, const void* d_in, int n_frames, float* d_H,
                          void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (n_frames == 0) return LSAS_OK;
  if (!d_in || !d_H) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  KParams k;
  base_params(p, &k);
  k.in = d_in;
  k.H_out = reinterpret_cast<float2*>(d_H);
  k.mode = kModeEstimate;
  k.use_tma = tma_ok(p, d_in) ? 1 : 0;
  const int grid = n_frames * k.chunks;
  ProfScope prof(p, "lsas_estimate", stream);
  if (p->launch(kKindEstimate, p->fmt == LSAS_IN_FC32, k, grid, p->geo.smem_est,
                static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status lsas_demodulate(lsas_plan p, const void* d_in, const float* d_H, int n_frames,
                            uint8_t* d_bits, float* d_eq, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (n_frames == 0) return LSAS_OK;
  if (!d_in || !d_H || !d_bits) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  ProfScope prof(p, "lsas_demodulate", stream);
  return launch_frame(p, d_in, n_frames, nullptr, d_H, d_bits, d_eq, kModeDemod,
                      static_cast<cudaStream_t>(stream));
}

lsas_status lsas_run_frame(lsas_plan p, const void* d_in, int n_frames, float* d_H,
                           uint8_t* d_bits, float* d_eq, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (n_frames == 0) return LSAS_OK;
  if (!d_in || !d_H || !d_bits) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  ProfScope prof(p, "lsas_run_frame", stream);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // whole waves of blocks run one frame per block; the frames after them may
  // run split into antenna shards (tail_shards)
  const int full = (n_frames / p->sms) * p->sms;
  const int G = tail_shards(p, n_frames - full);
  if (G == 1) return launch_frame(p, d_in, n_frames, d_H, nullptr, d_bits, d_eq, kModeRun, st);
  if (full > 0) {
    s = launch_frame(p, d_in, full, d_H, nullptr, d_bits, d_eq, kModeRun, st);
    if (s != LSAS_OK) return s;
  }
  return run_split_tail(p, d_in, full, n_frames - full, G, d_H, d_bits, d_eq, st);
}

lsas_status lsas_mrc_partial(lsas_plan p, const void* d_in, int n_frames, int m_begin,
                             int m_count, float* d_H, float* d_P, float* d_E, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (m_begin < 0 || m_count < 1 || m_begin > p->M - m_count) return LSAS_ERR_INVALID_ARG;
  if (n_frames == 0) return LSAS_OK;
  if (!d_in || !d_H || !d_P || !d_E) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  KParams k;
  base_params(p, &k);
  k.in = d_in;
  k.H_out = reinterpret_cast<float2*>(d_H);
  k.P_out = reinterpret_cast<float2*>(d_P);
  k.E_out = d_E;
  k.M = m_count;
  k.m0 = m_begin;
  k.chunks = (m_count + p->geo.Af - 1) / p->geo.Af;
  ProfScope prof(p, "lsas_mrc_partial", stream);
  k.mode = kModePartial;
  k.use_tma = tma_ok(p, d_in) ? 1 : 0;
  if (p->launch(kKindFrame, p->fmt == LSAS_IN_FC32, k, n_frames, p->geo.smem_frame,
                static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status lsas_mrc_combine(lsas_plan p, const float* d_P, const float* d_E, int n_shards,
                             int n_frames, uint8_t* d_bits, float* d_eq, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (n_shards < 1 || n_shards > 256) return LSAS_ERR_INVALID_ARG;
  if (n_frames == 0) return LSAS_OK;
  if (!d_P || !d_E || !d_bits) return LSAS_ERR_INVALID_ARG;
  // the kernel reads partials and energies 16 bytes at a time
  if ((reinterpret_cast<uintptr_t>(d_P) | reinterpret_cast<uintptr_t>(d_E)) % 16 != 0)
    return LSAS_ERR_INVALID_ARG;
  if (d_eq && reinterpret_cast<uintptr_t>(d_eq) % 8 != 0) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  KParams k;
  base_params(p, &k);
  k.P_in = reinterpret_cast<const float2*>(d_P);
  k.E_in = d_E;
  k.shards = n_shards;
  k.nframes = n_frames;
  k.bits = d_bits;
  k.eq = reinterpret_cast<float2*>(d_eq);
  ProfScope prof(p, "lsas_mrc_combine", stream);
  if (launch_combine(k, static_cast<cudaStream_t>(stream)) != cudaSuccess) return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status lsas_fft_tc(lsas_plan p, const void* d_in, int n_frames, int terms, float* d_Y,
                        void* stream) {
  return lsas_fft_tc_ex(p, d_in, n_frames, LSAS_TC_FP16, terms, d_Y, stream);
}

lsas_status lsas_fft_tc_ex(lsas_plan p, const void* d_in, int n_frames, int operand, int terms,
                           float* d_Y, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  if (terms != 1 && terms != 3) return LSAS_ERR_INVALID_ARG;
  if (operand != LSAS_TC_FP16 && operand != LSAS_TC_BF16) return LSAS_ERR_INVALID_ARG;
  if (!p->d_tc_w1 || p->fmt != LSAS_IN_SC16) return LSAS_ERR_UNSUPPORTED;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (n_frames == 0) return LSAS_OK;
  if (!d_in || !d_Y) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  KParams k;
  base_params(p, &k);
  k.in = d_in;
  k.Y_out = reinterpret_cast<float2*>(d_Y);
  k.nframes = n_frames;
  k.terms = terms;
  k.tc_bf16 = operand == LSAS_TC_BF16 ? 1 : 0;
  k.tc_w1 = p->d_tc_w1;
  k.tc_w2 = p->d_tc_w2;
  k.tc_tw = p->d_tc_tw;
  // one persistent block per SM (two when the shared memory allows)
  const size_t rows = static_cast<size_t>(n_frames) * p->M * p->S;
  const int per_batch = (128 / (p->N / 32) > 4) ? 128 / (p->N / 32) : 4;
  const size_t batches = (rows + per_batch - 1) / per_batch;
  const int per_sm = tc_smem_bytes(p->N) * 2 <= kSmemLimit ? 2 : 1;
  const size_t cap = static_cast<size_t>(p->sms) * per_sm;
  const int grid = static_cast<int>(batches < cap ? batches : cap);
  ProfScope prof(p, operand == LSAS_TC_BF16 ? "lsas_fft_tc_ex(bf16)" : "lsas_fft_tc", stream);
  if (launch_tcfft(k, p->N, grid, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status lsas_run_frame_refined(lsas_plan p, const void* d_in, int n_frames,
                                   const uint16_t* d_params_bf16, float* d_work, float* d_H,
                                   uint8_t* d_bits, float* d_eq, int* d_status, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  if (p->N != 1024 || p->fmt != LSAS_IN_SC16) return LSAS_ERR_UNSUPPORTED;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (n_frames == 0) return LSAS_OK;
  if (!d_in || !d_params_bf16 || !d_work || !d_H || !d_bits || !d_status)
    return LSAS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_work) % 16 != 0 || reinterpret_cast<uintptr_t>(d_in) % 4 != 0)
    return LSAS_ERR_INVALID_ARG;
  if (d_eq && reinterpret_cast<uintptr_t>(d_eq) % 8 != 0) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  ProfScope prof(p, "lsas_run_frame_refined", stream);
  KParams k;
  base_params(p, &k);
  k.in = d_in;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dn_ls_tc(k, d_params_bf16, n_frames, d_work, reinterpret_cast<float2*>(d_H), d_status,
               p->sms, st) != cudaSuccess)
    return LSAS_ERR_CUDA;
  return launch_frame(p, d_in, n_frames, nullptr, d_H, d_bits, d_eq, kModeDemod, st);
}

lsas_status lsas_receive_y(lsas_plan p, const float* d_Y, int n_frames, float* d_H,
                           uint8_t* d_bits, float* d_eq, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (n_frames == 0) return LSAS_OK;
  if (!d_Y || !d_H || !d_bits) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  KParams k;
  base_params(p, &k);
  k.Y_out = reinterpret_cast<float2*>(const_cast<float*>(d_Y));
  k.H_out = reinterpret_cast<float2*>(d_H);
  k.bits = d_bits;
  k.eq = reinterpret_cast<float2*>(d_eq);
  ProfScope prof(p, "lsas_receive_y", stream);
  if (launch_yrx(k, n_frames, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status lsas_plan_set_pn(lsas_plan p, const float* host_pn, int len) {
  if (!p || !host_pn || len < 1 || len > kMaxPnLen) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  if (!p->d_pn && cudaMalloc(&p->d_pn, sizeof(float) * kMaxPnLen) != cudaSuccess) {
    cudaGetLastError();
    return LSAS_ERR_OOM;
  }
  if (cudaMemcpy(p->d_pn, host_pn, sizeof(float) * len, cudaMemcpyHostToDevice) != cudaSuccess)
    return LSAS_ERR_CUDA;
  p->pn_len = len;
  return LSAS_OK;
}

lsas_status lsas_pn_sync(lsas_plan p, const void* d_capture, int n_frames, int capture_len,
                         int window, int* d_offset, float* d_peak, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  if (p->pn_len < 1) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (window < 1 || capture_len < 1 || window > capture_len - p->pn_len + 1)
    return LSAS_ERR_INVALID_ARG;
  if (n_frames == 0) return LSAS_OK;
  if (!d_capture || !d_offset) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  KParams k;
  base_params(p, &k);
  k.in = d_capture;
  k.pn = p->d_pn;
  k.pn_len = p->pn_len;
  k.cap_len = capture_len;
  k.window = window;
  k.offsets = d_offset;
  k.peaks = d_peak;
  ProfScope prof(p, "lsas_pn_sync", stream);
  if (launch_pn(k, p->fmt == LSAS_IN_FC32, n_frames, static_cast<cudaStream_t>(stream)) !=
      cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status lsas_pn_extract(lsas_plan p, const void* d_capture, int n_frames, int capture_len,
                            const int* d_offset, int backoff, void* d_frames, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (capture_len < 1 || backoff < 0) return LSAS_ERR_INVALID_ARG;
  if (n_frames == 0) return LSAS_OK;
  if (!d_capture || !d_offset || !d_frames) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  KParams k;
  base_params(p, &k);
  k.in = d_capture;
  k.offsets_in = d_offset;
  k.pn_len = p->pn_len;
  k.backoff = backoff;
  k.cap_len = capture_len;
  k.Y_out = static_cast<float2*>(d_frames);
  ProfScope prof(p, "lsas_pn_extract", stream);
  if (launch_extract(k, p->fmt == LSAS_IN_FC32, n_frames, static_cast<cudaStream_t>(stream)) !=
      cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status lsas_fftshift(lsas_plan p, int what, void* d_buf, int n_frames, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  size_t rows = 0;
  switch (what) {
    case LSAS_SHIFT_H: rows = static_cast<size_t>(n_frames) * p->M; break;
    case LSAS_SHIFT_EQ: rows = static_cast<size_t>(n_frames) * p->D; break;
    case LSAS_SHIFT_Y: rows = static_cast<size_t>(n_frames) * p->M * p->S; break;
    case LSAS_SHIFT_BITS: rows = static_cast<size_t>(n_frames) * p->D; break;
    default: return LSAS_ERR_INVALID_ARG;
  }
  if (n_frames == 0) return LSAS_OK;
  if (!d_buf) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  const int kind = what == LSAS_SHIFT_BITS ? 1 : 0;
  ProfScope prof(p, "lsas_fftshift", stream);
  if (launch_shift(d_buf, kind, rows, p->N, p->N * p->q / 8, p->sms,
                   static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status lsas_plan_set_fault(lsas_plan p, int kind) {
  if (!p || kind < 0 || kind > 1) return LSAS_ERR_INVALID_ARG;
  p->fault = kind;
  return LSAS_OK;
}

lsas_status lsas_plan_device_bytes(lsas_plan p, size_t* out_bytes) {
  if (!p || !out_bytes) return LSAS_ERR_INVALID_ARG;
  *out_bytes = p->dev_bytes;
  return LSAS_OK;
}

lsas_status lsas_plan_set_batch_split(lsas_plan p, int enable) {
  if (!p || enable < 0 || enable > 2) return LSAS_ERR_INVALID_ARG;
  p->batch_split = enable;
  return LSAS_OK;
}

lsas_status lsas_plan_batch_split_shards(lsas_plan p, int n_frames, int* out_shards) {
  if (!p || !out_shards || n_frames < 0) return LSAS_ERR_INVALID_ARG;
  *out_shards = tail_shards(p, n_frames - (n_frames / p->sms) * p->sms);
  return LSAS_OK;
}

lsas_status lsas_run_frame_host(lsas_plan p, const void* h_in, int n_frames, float* h_H,
                                uint8_t* h_bits, float* h_eq, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (n_frames == 0) return LSAS_OK;
  if (!h_in || !h_H || !h_bits) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  const int chunk = p->max_frames < kHostChunk ? p->max_frames : kHostChunk;
  const size_t inb = in_bytes_per_frame(p->M, p->N, p->cp, p->S, p->fmt);
  const size_t hb = static_cast<size_t>(p->M) * p->N * 8;
  const size_t bb = bits_bytes_per_frame(p->N, p->S, p->Q);
  const size_t eb = static_cast<size_t>(p->D) * p->N * 8;
  // The receiver never reads the cyclic prefixes (step 1 drops them), so a
  // pitched copy moves only the N samples after each prefix once rows are
  // long enough for pitched copies to run at full speed; the staging buffer
  // keeps the [M][S*(N+CP)] layout.
  const size_t bps = p->fmt == LSAS_IN_SC16 ? 4 : 8;
  const size_t pitch = static_cast<size_t>(p->N + p->cp) * bps;
  const size_t keep = static_cast<size_t>(p->N) * bps, skip = static_cast<size_t>(p->cp) * bps;
  const bool strip = host_strips_cp(p->N, p->cp, p->fmt);
  if (!p->d_in_stage[0]) {
    for (int i = 0; i < 2; ++i) {
      if (cudaMalloc(&p->d_in_stage[i], inb * chunk) != cudaSuccess ||
          cudaMalloc(&p->d_H_stage[i], hb * chunk) != cudaSuccess ||
          cudaMalloc(&p->d_bits_stage[i], bb * chunk) != cudaSuccess ||
          cudaMalloc(&p->d_eq_stage[i], eb * chunk) != cudaSuccess) {
        cudaGetLastError();
        return LSAS_ERR_OOM;
      }
    }
    if (cudaStreamCreateWithFlags(&p->up_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->down_stream, cudaStreamNonBlocking) != cudaSuccess)
      return LSAS_ERR_CUDA;
    for (int i = 0; i < 2; ++i)
      if (cudaEventCreateWithFlags(&p->ev_up[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&p->ev_k[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&p->ev_down[i], cudaEventDisableTiming) != cudaSuccess)
        return LSAS_ERR_CUDA;
  }
  ProfScope prof(p, "lsas_run_frame_host", stream, /*host=*/true);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Chunk c uses staging buffer c % 2.  Uploads run on up_stream, kernels on
  // the caller's stream, downloads on down_stream, so the upload of chunk
  // c+1 and the download of chunk c-1 overlap the kernel of chunk c.  The
  // upload into a buffer waits for the download of the chunk that used it
  // last, which itself waited for that chunk's kernel.
  const int nchunks = (n_frames + chunk - 1) / chunk;
  for (int c = 0; c < nchunks; ++c) {
    const int b = c % 2;
    const int f0 = c * chunk;
    const int nf = (n_frames - f0) < chunk ? (n_frames - f0) : chunk;
    if (c >= 2 && cudaStreamWaitEvent(p->up_stream, p->ev_down[b], 0) != cudaSuccess)
      return LSAS_ERR_CUDA;
    const unsigned char* src = static_cast<const unsigned char*>(h_in) + inb * f0;
    unsigned char* dst = static_cast<unsigned char*>(p->d_in_stage[b]);
    const cudaError_t up =
        strip ? cudaMemcpy2DAsync(dst + skip, pitch, src + skip, pitch, keep,
                                  static_cast<size_t>(p->M) * p->S * nf, cudaMemcpyHostToDevice,
                                  p->up_stream)
              : cudaMemcpyAsync(dst, src, inb * nf, cudaMemcpyHostToDevice, p->up_stream);
    if (up != cudaSuccess || cudaEventRecord(p->ev_up[b], p->up_stream) != cudaSuccess ||
        cudaStreamWaitEvent(st, p->ev_up[b], 0) != cudaSuccess)
      return LSAS_ERR_CUDA;
    lsas_status r = launch_frame(p, p->d_in_stage[b], nf, reinterpret_cast<float*>(p->d_H_stage[b]),
                                 nullptr, p->d_bits_stage[b],
                                 h_eq ? reinterpret_cast<float*>(p->d_eq_stage[b]) : nullptr,
                                 kModeRun, st);
    if (r != LSAS_OK) return r;
    if (cudaEventRecord(p->ev_k[b], st) != cudaSuccess ||
        cudaStreamWaitEvent(p->down_stream, p->ev_k[b], 0) != cudaSuccess)
      return LSAS_ERR_CUDA;
    if (cudaMemcpyAsync(h_H + hb / 4 * f0, p->d_H_stage[b], hb * nf, cudaMemcpyDeviceToHost,
                        p->down_stream) != cudaSuccess ||
        cudaMemcpyAsync(h_bits + bb * f0, p->d_bits_stage[b], bb * nf, cudaMemcpyDeviceToHost,
                        p->down_stream) != cudaSuccess)
      return LSAS_ERR_CUDA;
    if (h_eq && cudaMemcpyAsync(h_eq + eb / 4 * f0, p->d_eq_stage[b], eb * nf,
                                cudaMemcpyDeviceToHost, p->down_stream) != cudaSuccess)
      return LSAS_ERR_CUDA;
    if (cudaEventRecord(p->ev_down[b], p->down_stream) != cudaSuccess) return LSAS_ERR_CUDA;
  }
  if (cudaStreamSynchronize(p->down_stream) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LSAS_ERR_CUDA;
  return LSAS_OK;
}

lsas_status lsas_plan_sync(lsas_plan p, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LSAS_ERR_CUDA;
  int st = 0;
  if (cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess)
    return LSAS_ERR_CUDA;
  return static_cast<lsas_status>(st);
}

lsas_status lsas_plan_info(lsas_plan p, int out[8]) {
  if (!p || !out) return LSAS_ERR_INVALID_ARG;
  out[0] = p->geo.Af;
  out[1] = p->geo.T;
  out[2] = p->geo.smem_frame;
  out[3] = p->geo.groups;
  out[4] = p->geo.nslots;
  const int bps = p->fmt == LSAS_IN_SC16 ? 4 : 8;
  out[5] = (((p->N + p->cp) * bps) % 16 == 0 && (p->cp * bps) % 16 == 0) ? 1 : 0;
  out[6] = static_cast<int>(p->fmt);
  out[7] = p->max_frames;
  return LSAS_OK;
}

lsas_status lsas_plan_set_profile(lsas_plan p, int on) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(p->prof_mu);
  p->prof = on != 0;
  return LSAS_OK;
}

lsas_status lsas_plan_profile(lsas_plan p, char* buf, size_t len, size_t* needed) {
  if (!p || (!buf && !needed)) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(p->prof_mu);
  // fold the finished records (waits for the calls' stop events)
  lsas_status st = LSAS_OK;
  for (const auto& r : p->prof_recs) {
    double ms = r.host_ms;
    if (r.a) {
      float f = 0.f;
      if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&f, r.a, r.b) != cudaSuccess) {
        cudaGetLastError();
        st = LSAS_ERR_CUDA;
      }
      ms = f;
      p->prof_pool.push_back(r.a);
      p->prof_pool.push_back(r.b);
    }
    auto& acc = p->prof_acc[r.name];
    acc.first += 1;
    acc.second += ms;
  }
  p->prof_recs.clear();
  if (st != LSAS_OK) return st;
  std::string js = "{";
  char item[192];
  bool first = true;
  for (const auto& kv : p->prof_acc) {
    std::snprintf(item, sizeof(item), "%s\"%s\": {\"calls\": %llu, \"ms\": %.6f}", first ? "" : ", ",
                  kv.first.c_str(), static_cast<unsigned long long>(kv.second.first), kv.second.second);
    js += item;
    first = false;
  }
  js += "}";
  if (needed) *needed = js.size() + 1;
  if (!buf) return LSAS_OK;
  if (len < js.size() + 1) return LSAS_ERR_CAPACITY;
  std::memcpy(buf, js.c_str(), js.size() + 1);
  p->prof_acc.clear();
  return LSAS_OK;
}

lsas_status lsas_plan_destroy(lsas_plan p) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) == LSAS_OK) cudaDeviceSynchronize();
  cudaFree(p->d_twP);
  cudaFree(p->d_xinv);
  cudaFree(p->d_status);
  cudaFree(p->d_tc_w1);
  cudaFree(p->d_tc_w2);
  cudaFree(p->d_tc_tw);
  cudaFree(p->d_pn);
  cudaFree(p->d_tail);
  if (p->tail_ev) cudaEventDestroy(p->tail_ev);
  for (int i = 0; i < 2; ++i) {
    cudaFree(p->d_in_stage[i]);
    cudaFree(p->d_H_stage[i]);
    cudaFree(p->d_bits_stage[i]);
    cudaFree(p->d_eq_stage[i]);
  }
  if (p->up_stream) cudaStreamDestroy(p->up_stream);
  if (p->down_stream) cudaStreamDestroy(p->down_stream);
  for (int i = 0; i < 2; ++i) {
    if (p->ev_up[i]) cudaEventDestroy(p->ev_up[i]);
    if (p->ev_k[i]) cudaEventDestroy(p->ev_k[i]);
    if (p->ev_down[i]) cudaEventDestroy(p->ev_down[i]);
  }
  for (const auto& r : p->prof_recs) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : p->prof_pool) cudaEventDestroy(e);
  delete p;
  return LSAS_OK;
}

lsas_status lsas_run_frame_split_static(lsas_plan p, const void* d_in, int n_frames,
                                        int n_shards, float* d_H, uint8_t* d_bits,
                                        float* d_eq, void* stream) {
  if (!p) return LSAS_ERR_INVALID_ARG;
  if (n_shards < 1 || n_shards > p->M || n_frames < 0) return LSAS_ERR_INVALID_ARG;
  // partial sums of every shard and frame: P [G][F][D][N] complex, then E [G][F][N]
  const size_t p_bytes = static_cast<size_t>(n_shards) * n_frames * p->D * p->N * 8;
  const size_t e_bytes = static_cast<size_t>(n_shards) * n_frames * p->N * 4;
  if (p_bytes + e_bytes > LSAS_STATIC_SCRATCH_BYTES) return LSAS_ERR_CAPACITY;
  lsas_status s = check_frames(p, n_frames);
  if (s != LSAS_OK) return s;
  if (n_frames == 0) return LSAS_OK;
  if (!d_in || !d_H || !d_bits) return LSAS_ERR_INVALID_ARG;
  // everything the combine pass would reject is rejected here, before the
  // shard pass is launched
  if (d_eq && reinterpret_cast<uintptr_t>(d_eq) % 8 != 0) return LSAS_ERR_INVALID_ARG;
  if (set_device(p) != LSAS_OK) return LSAS_ERR_CUDA;
  ProfScope prof(p, "lsas_run_frame_split_static", stream);
  unsigned char* scratch = static_cast<unsigned char*>(p->d_split_scratch);
  if (!scratch) return LSAS_ERR_CUDA;
  float* P = reinterpret_cast<float*>(scratch);
  float* E = reinterpret_cast<float*>(scratch + p_bytes);   // p_bytes is a multiple of 512
  if (p->M % n_shards == 0 && n_shards > 1) {
    // equal shards: one launch, grid row g = shard g, so the shards of a
    // frame run side by side (the same partial sums as one launch per shard)
    KParams k;
    base_params(p, &k);
    k.in = d_in;
    k.H_out = reinterpret_cast<float2*>(d_H);
    k.P_out = reinterpret_cast<float2*>(P);
    k.E_out = E;
    k.M = p->M / n_shards;
    k.shard_y = k.M;
    k.grid_y = n_shards;
    // small batches: one block per data-symbol group as well (each repeats
    // the pilot transform), so a frame's groups also run side by side
    k.group_z = ((p->N <= 1024 || p->fmt == LSAS_IN_SC16) && p->geo.groups > 1 &&
                 n_frames * n_shards * 2 <= p->sms) ? 1 : 0;
    k.chunks = (k.M + p->geo.Af - 1) / p->geo.Af;
    k.mode = kModePartial;
    k.use_tma = tma_ok(p, d_in) ? 1 : 0;
    if (p->launch(kKindFrame, p->fmt == LSAS_IN_FC32, k, n_frames, p->geo.smem_frame,
                  static_cast<cudaStream_t>(stream)) != cudaSuccess)
      return LSAS_ERR_CUDA;
    return lsas_mrc_combine(p, P, E, n_shards, n_frames, d_bits, d_eq, stream);
  }
  // even split: shard g gets M / G antennas, plus one for the first M % G shards
  int m0 = 0;
  for (int g = 0; g < n_shards; ++g) {
    const int mc = p->M / n_shards + (g < p->M % n_shards ? 1 : 0);
    s = lsas_mrc_partial(p, d_in, n_frames, m0, mc, d_H,
                         P + static_cast<size_t>(g) * n_frames * p->D * p->N * 2,
                         E + static_cast<size_t>(g) * n_frames * p->N, stream);
    if (s != LSAS_OK) return s;
    m0 += mc;
  }
  return lsas_mrc_combine(p, P, E, n_shards, n_frames, d_bits, d_eq, stream);
}

}  // extern "C"
