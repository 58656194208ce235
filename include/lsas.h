/*
 * lsas.h -- C ABI of liblsas: LS channel estimation and MRC demodulation of
 * uplink OFDM frames for large-scale antenna receivers, on one GB300 GPU.
 *
 * The operations are those of the paper "Accelerating Channel Estimation and
 * Demodulation of Uplink OFDM symbols for Large Scale Antenna Systems using
 * GPU" (arXiv 1901.07499):
 *   - cyclic-prefix removal and an N-point FFT of every OFDM symbol of every
 *     receive antenna (Sec. II-B, Sec. II-C: batched FFTs over antennas);
 *   - block-type Least Squares estimation from the first (pilot) symbol,
 *     H[m,k] = Y_pilot[m,k] / X_pilot[k] (Sec. II-B, Sec. II-C);
 *   - Maximal Ratio Combining of each data symbol over the M antennas with the
 *     conjugate channel and the channel-energy sum formed once per frame
 *     (Sec. II-C, Sec. III);
 *   - hard decision of the combined symbols to Gray-labelled QAM bits (the
 *     demodulated output of Sec. II-B).
 * The paper calls the antenna count N and the subcarrier count M; this ABI
 * uses M = antennas and N = FFT length = subcarriers throughout.
 *
 * Conventions fixed by this library where the paper leaves them open:
 *   - forward FFT kernel exp(-2j pi k n / N), unitary scale 1/sqrt(N);
 *     subcarriers in natural order k = 0 .. N-1 (lsas_fftshift reorders
 *     outputs the way the paper does);
 *   - LS for a general pilot: H = Y conj(X) / |X|^2;
 *   - normalised MRC: z[d,k] = sum_m conj(H[m,k]) Y[m,d,k] / sum_m |H[m,k]|^2;
 *   - square Gray QAM of unit average energy: per axis L = sqrt(Q) levels at
 *     (2i - (L-1)) A, A = 1/sqrt(2(Q-1)/3); the level of a value v is the
 *     number of boundaries (2b - L) A, b = 1..L-1, with v >= boundary (a value
 *     on a boundary goes to the upper level), compared in float32; level i
 *     carries the Gray word i ^ (i >> 1), MSB first, I-axis bits before
 *     Q-axis bits.  BPSK (Q = 2) uses the I axis only, boundary 0.
 *
 * Buffers (all contiguous, row-major; "d_" = device memory, "h_" = host):
 *   input  [F][M][S*(N+CP)] interleaved IQ samples: int16 pairs (SC16, the
 *          value is used as is, no rescaling) or float32 pairs (FC32)
 *   H      [F][M][N]  complex float32 (re, im interleaved)
 *   Y      [F][M][S][N] complex float32 (lsas_fft only)
 *   eq     [F][D][N]  complex float32, the combined symbols z (optional)
 *   bits   [F][D*N*q/8] bytes; bit t = (d*N + k)*q + j of a frame is bit
 *          (7 - t%8) of byte t/8 (MSB first), d = data-symbol index in
 *          ascending symbol order skipping the pilot, j = bit of the symbol.
 * with F frames, M antennas, N subcarriers, S symbols per frame (one pilot
 * at pilot_idx, D = S - 1 data symbols), q = log2(Q) bits per data symbol.
 *
 * Ownership: the caller owns every buffer passed in.  A plan owns only its own
 * device tables (twiddles, pilot inverse, a status word) and, after the first
 * lsas_run_frame_host call, its host-transfer staging buffers.
 *
 * Errors: argument checks run on the host before any launch; a failing check
 * returns its code and enqueues nothing.  A CUDA launch or copy failure
 * returns LSAS_ERR_CUDA.  Conditions found on the device (a zero or non-finite
 * channel energy, a wait that timed out) are latched into the plan's status
 * word and returned by lsas_plan_sync.  Calls on one plan from several host
 * threads at once are not supported.
 */
#ifndef LSAS_H_
#define LSAS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsas_plan_s* lsas_plan;

typedef enum {
  LSAS_OK = 0,
  LSAS_ERR_INVALID_ARG = 1,  /* bad size, null pointer, misuse */
  LSAS_ERR_UNSUPPORTED = 2,  /* valid request this build does not handle */
  LSAS_ERR_OOM = 3,          /* device or pinned-host allocation failed */
  LSAS_ERR_CAPACITY = 4,     /* n_frames above the plan's max_frames */
  LSAS_ERR_CUDA = 5,         /* a CUDA runtime call failed */
  LSAS_ERR_TIMEOUT = 6,      /* a bounded device wait gave up (latched) */
  LSAS_ERR_DEVICE = 7        /* zero / non-finite channel energy (latched) */
} lsas_status;

typedef enum { LSAS_IN_SC16 = 0, LSAS_IN_FC32 = 1 } lsas_input_fmt;

/* Human-readable name of a status code (static string, never NULL). */
const char* lsas_status_str(lsas_status s);

/*
 * Host-only check of a receiver configuration; touches no GPU.
 * Supported: 1 <= M <= 256; N a power of two in [64, 2048];
 * 0 <= cp_len < N; 2 <= n_sym <= 64; 0 <= pilot_idx < n_sym;
 * qam_order in {2, 4, 16, 64, 256}.  Returns LSAS_OK or LSAS_ERR_INVALID_ARG.
 */
lsas_status lsas_check_config(int M, int N, int cp_len, int n_sym,
                              int pilot_idx, int qam_order);

/*
 * Host-only: bytes per frame of the input (for fmt), of H, of the packed bits
 * and of eq, written to out[0..3].  Returns LSAS_ERR_INVALID_ARG for a bad
 * configuration or a NULL out.
 */
lsas_status lsas_frame_bytes(int M, int N, int cp_len, int n_sym,
                             int qam_order, lsas_input_fmt fmt,
                             size_t out[4]);

/*
 * Create a plan on the current CUDA device: validates the configuration (as
 * lsas_check_config), uploads the twiddle table and the default all-(+1)
 * pilot, and prepares the kernels.  Defaults: SC16 input, max_frames = 1024.
 * On success *out holds the plan; on failure *out is set to NULL.
 */
lsas_status lsas_plan_create(int M, int N, int cp_len, int n_sym,
                             int pilot_idx, int qam_order, lsas_plan* out);

/* Select the input sample format and the largest n_frames a call accepts. */
lsas_status lsas_plan_set(lsas_plan plan, lsas_input_fmt fmt, int max_frames);

/*
 * Set the known pilot symbol X_pilot[k] (Sec. II-B channel-estimation
 * symbol) from N interleaved (re, im) float pairs in host memory.  Every
 * |X[k]| must be non-zero and finite, else LSAS_ERR_INVALID_ARG.
 * Synchronous (the table is uploaded before return).
 */
lsas_status lsas_plan_set_pilot(lsas_plan plan, const float* host_pilot_iq);

/*
 * CP removal + unitary FFT of every symbol of every antenna (Sec. II-B,
 * Sec. II-C): d_Y[f][m][s][k] = N^-1/2 sum_n r[f][m][s][n] exp(-2j pi k n/N).
 * Asynchronous on stream (a cudaStream_t; NULL = legacy default stream).
 */
lsas_status lsas_fft(lsas_plan plan, const void* d_in, int n_frames,
                     float* d_Y, void* stream);

/*
 * LS channel estimation from the pilot symbol (Sec. II-C):
 * d_H[f][m][k] = Y[f][m][pilot_idx][k] conj(X[k]) / |X[k]|^2.  Asynchronous.
 */
lsas_status lsas_estimate(lsas_plan plan, const void* d_in, int n_frames,
                          float* d_H, void* stream);

/*
 * MRC demodulation of the data symbols with a given channel d_H (Sec. II-C):
 * writes d_bits and, if d_eq is not NULL, the combined symbols z.  d_H may
 * come from lsas_estimate or from any other estimator.  Asynchronous.
 */
lsas_status lsas_demodulate(lsas_plan plan, const void* d_in,
                            const float* d_H, int n_frames, uint8_t* d_bits,
                            float* d_eq, void* stream);

/*
 * The whole receiver in one fused pass per frame: estimation (writes d_H)
 * then demodulation (writes d_bits and optionally d_eq).  Asynchronous.
 * Whole waves of frames (one frame per SM) run in one launch.  The frames
 * after the last whole wave, or all of them for a batch smaller than one
 * wave, may run split into equal antenna shards so that they occupy more
 * SMs: the shards' MRC partial sums go to a scratch array the plan owns
 * (lsas_plan_create reserves at most 96 MiB for it), and the combine pass
 * forms z and the bits from them, summing the shards in a fixed order.
 * Outputs agree with the unsplit pass to rounding (the antenna sums are
 * ordered differently).  Calls on one plan from several streams take turns
 * on the scratch array: a split waits for the previous split's combine.
 * lsas_plan_set_batch_split turns the split off.
 */
lsas_status lsas_run_frame(lsas_plan plan, const void* d_in, int n_frames,
                           float* d_H, uint8_t* d_bits, float* d_eq,
                           void* stream);

/*
 * Antenna split, shard step (the distributed receiver of Sec. IV: MRC of
 * Sec. II-C separates over antennas).  Runs the fused receiver for antennas
 * [m_begin, m_begin + m_count) of the plan's M and stops at the MRC sums:
 *   d_H  [F][M][N] complex: rows m_begin .. m_begin+m_count-1 are written
 *        (the LS estimate, as lsas_run_frame writes them), others untouched;
 *   d_P  [F][D][N] complex: P[d][k] = sum over the shard of
 *        conj(H[m][k]) Y[m][s_d][k] (unitary Y);
 *   d_E  [F][N] float: E[k] = sum over the shard of |H[m][k]|^2.
 * d_in is the plan's [F][M][S*(N+CP)] input; only the shard's rows are read.
 * A device that holds only its own antennas uses a plan with M = its count,
 * m_begin = 0, m_count = M.  Errors: INVALID_ARG for a null pointer or a range
 * outside [0, M); CAPACITY for n_frames > max_frames.  Asynchronous.
 */
lsas_status lsas_mrc_partial(lsas_plan plan, const void* d_in, int n_frames,
                             int m_begin, int m_count, float* d_H, float* d_P,
                             float* d_E, void* stream);

/*
 * Antenna split, combine step: adds the partials of n_shards shards in shard
 * order 0 .. n_shards-1, then z = P / E, Gray slicing and packed bits exactly
 * as lsas_run_frame.  d_P is [n_shards][F][D][N] complex and d_E
 * [n_shards][F][N] float (shard g's lsas_mrc_partial outputs, stacked), both
 * 16-byte aligned; d_bits [F][ceil(D*N*q/8)]; d_eq [F][D][N] complex or NULL.
 * Only N, S, pilot position and QAM order of the plan matter here (not M).
 * Zero or non-finite summed energy gives z = 0 and latches LSAS_ERR_DEVICE.
 * Errors: INVALID_ARG for null/misaligned pointers or n_shards outside
 * [1, 256]; CAPACITY for n_frames > max_frames.  Asynchronous.
 */
lsas_status lsas_mrc_combine(lsas_plan plan, const float* d_P, const float* d_E,
                             int n_shards, int n_frames, uint8_t* d_bits,
                             float* d_eq, void* stream);

/*
 * Steps a1-a2 (CP removal + FFT, Sec. II-B/II-C) on the tensor cores: the
 * N-point DFT as two batched DFT-factor GEMMs (N = 32 x N/32, a twiddle
 * between them) on tcgen05 with fp16 operands and fp32 accumulation in
 * tensor memory.  terms = 3 splits every operand into fp16 hi + lo parts and
 * sums three products (relative error ~1e-6); terms = 1 uses plain fp16
 * operands (~1e-3).  Output as lsas_fft: d_Y [F][M][S][N] complex, unitary.
 * A precision form of the FFT, next to the FP32 path lsas_fft.
 * Supported: N in {512, 1024, 2048} and sc16 input, else LSAS_ERR_UNSUPPORTED;
 * terms other than 1 or 3 give LSAS_ERR_INVALID_ARG.  Asynchronous.
 */
lsas_status lsas_fft_tc(lsas_plan plan, const void* d_in, int n_frames, int terms,
                        float* d_Y, void* stream);

/*
 * lsas_fft_tc with a choice of operand type (Sec. II-C, the batched FFT as
 * DFT-factor GEMMs): operand LSAS_TC_FP16 (lsas_fft_tc itself) or
 * LSAS_TC_BF16, bfloat16 operands with fp32 accumulation.  terms = 1 uses
 * each operand rounded once (bf16: 8 significant bits, ~1e-2 relative
 * error); terms = 3 splits every operand into hi = round(v) and
 * lo = round(v - hi) of the same type and sums a_hi b_hi + a_hi b_lo +
 * a_lo b_hi (bf16: ~2^-16 relative).  The constant DFT operands of both
 * types are tables the plan builds in double precision.  INVALID_ARG for
 * another operand or terms; otherwise as lsas_fft_tc.
 */
#define LSAS_TC_FP16 0
#define LSAS_TC_BF16 1
lsas_status lsas_fft_tc_ex(lsas_plan plan, const void* d_in, int n_frames, int operand,
                           int terms, float* d_Y, void* stream);

/*
 * Steps a3-a5 from transformed symbols (the staged form of the receiver):
 * d_Y [F][M][S][N] complex (unitary FFT outputs, as lsas_fft or lsas_fft_tc
 * write them) -> LS estimate d_H [F][M][N] (Sec. II-C), MRC over the
 * antennas in antenna order and the Gray slicer, exactly the outputs of
 * lsas_run_frame (d_bits, optional d_eq).  Zero channel energy latches
 * LSAS_ERR_DEVICE.  Asynchronous.
 */
lsas_status lsas_receive_y(lsas_plan plan, const float* d_Y, int n_frames, float* d_H,
                           uint8_t* d_bits, float* d_eq, void* stream);

/*
 * Packet detection (Sec. II-B): the receiver correlates the received
 * baseband with the maximum-length PN sequence that precedes every frame to
 * find where the packet begins.  lsas_plan_set_pn stores the real PN chips
 * (host array of len floats, 1 <= len <= 1024; the plan copies them).
 */
lsas_status lsas_plan_set_pn(lsas_plan plan, const float* host_pn, int len);

/*
 * For every frame f of d_capture [F][M][capture_len] (interleaved IQ in the
 * plan's input format), the preamble start
 *   d_offset[f] = argmax over tau < window of
 *                 sum_m |sum_n pn[n] y[f][m][tau + n]|^2
 * (the earliest tau on ties) and, if d_peak is not NULL, d_peak[f] = that
 * maximum (float).  The frame begins at d_offset[f] + len.  Errors:
 * INVALID_ARG if no PN sequence is set, for window < 1 or
 * window + len - 1 > capture_len, or a null pointer; CAPACITY for
 * n_frames > max_frames.  Asynchronous.
 */
lsas_status lsas_pn_sync(lsas_plan plan, const void* d_capture, int n_frames,
                         int capture_len, int window, int* d_offset,
                         float* d_peak, void* stream);

/*
 * Copy each frame out of its capture into the receiver's input layout:
 * d_frames [F][M][S*(N+CP)] (plan format) takes the S*(N+CP) samples of each
 * antenna row from d_offset[f] + len - backoff.  A backoff of a few samples
 * starts the FFT windows early inside the cyclic prefix, which the LS
 * estimate absorbs as a phase ramp; a late start would take samples of the
 * next symbol.  A start outside the capture zero-fills that frame and
 * latches LSAS_ERR_DEVICE.  Errors: INVALID_ARG for backoff < 0 or a null
 * pointer; CAPACITY for n_frames > max_frames.  Asynchronous.
 */
lsas_status lsas_pn_extract(lsas_plan plan, const void* d_capture, int n_frames,
                            int capture_len, const int* d_offset, int backoff,
                            void* d_frames, void* stream);

/*
 * fftshift (Sec. II-C): reorder the subcarriers of an output buffer in place
 * so that subcarrier k moves to (k + N/2) mod N (the zero-frequency bin to
 * the middle).  what selects the buffer and its layout:
 *   LSAS_SHIFT_H    d_buf [F][M][N] complex      LSAS_SHIFT_EQ  [F][D][N] complex
 *   LSAS_SHIFT_Y    [F][M][S][N] complex         LSAS_SHIFT_BITS [F][D][N*q/8] bytes
 * Applying it twice restores the natural order.  Errors: INVALID_ARG for an
 * unknown what or a null pointer; CAPACITY for n_frames > max_frames.
 */
enum { LSAS_SHIFT_H = 0, LSAS_SHIFT_EQ = 1, LSAS_SHIFT_Y = 2, LSAS_SHIFT_BITS = 3 };
lsas_status lsas_fftshift(lsas_plan plan, int what, void* d_buf, int n_frames,
                          void* stream);

/*
 * Serving loop.  The paper processes frames as they arrive from the radios
 * (Sec. II-B) and names frame-level batching as its next step (Sec. IV).  A
 * server takes frames of several registered receiver configurations, one at
 * a time, from host memory, batches them per configuration and runs the
 * fused receiver (lsas_run_frame) on each batch.  Each configuration has two
 * lanes (a stream with staging for max_batch frames) and at most one batch
 * per lane in flight.  While both are busy its frames wait and the next
 * batch takes up to max_batch of them.
 *
 * lsas_server_create: memory budget in bytes for everything registered
 *   later; max_batch frames per launch (1..1024); max_wait_us, how long the
 *   oldest waiting frame of a configuration may wait for more frames of it.
 *   Starts one worker thread on the current device.  CUDA if there is no
 *   device, INVALID_ARG for bad arguments.
 * lsas_server_register: admit a configuration (as lsas_plan_create, plus the
 *   input format and an optional host pilot of N interleaved re,im floats).
 *   Its plan and the staging of both lanes (2 * max_batch frames) count
 *   against the budget: LSAS_ERR_CAPACITY when they do not fit.  Returns
 *   its id.
 * lsas_server_register_refined: as lsas_server_register, for the learned
 *   form of the receiver: each batch runs LS (lsas_estimate), the
 *   tensor-core refinement (lsas_dn_apply_tc with d_params_bf16, a device
 *   array of LSAS_DN_PARAMS bf16 values that must stay valid until the
 *   server is destroyed) and MRC + demap with the refined channel
 *   (lsas_demodulate); h_H receives the refined channel.  N must be a
 *   multiple of 128 (UNSUPPORTED otherwise).  The LS estimate and the
 *   refinement's scratch of both lanes count against the budget too.
 * lsas_server_set_admission: per-frame memory admission.  Every submitted
 *   frame is charged its device footprint (input, H, bits and, when h_eq is
 *   given, z bytes per frame) from submission until its results are home.
 *   Frames are admitted while the charged total stays within
 *   frame_budget_bytes (0, the default: what the memory budget leaves after
 *   registration).  A frame that does not fit is refused with
 *   LSAS_ERR_CAPACITY at once (wait_ms = 0, the default) or after waiting up
 *   to wait_ms for frames to complete.  INVALID_ARG for a null server or a
 *   negative wait.
 * lsas_server_frame_bytes: out[0] bytes charged by frames queued or in
 *   flight, out[1] the frame budget in force.
 * lsas_server_submit: queue one frame of a registered configuration:
 *   h_in [M][S*(N+CP)] samples, results to h_H [M][N], h_bits [D*N*q/8],
 *   h_eq [D][N] (nullable), all host memory that stays valid until the wait
 *   returns (pinned memory for full copy speed).  Admission as above
 *   (LSAS_ERR_CAPACITY when the frame does not fit); gives a ticket.
 * lsas_server_wait: wait up to timeout_ms for a ticket's results;
 *   LSAS_ERR_TIMEOUT if they are not ready (the ticket stays valid),
 *   INVALID_ARG for an unknown ticket.  latency_us (nullable) receives the
 *   time from submit to results in host memory.
 * lsas_server_submit_many: lsas_server_submit for n frames in one call
 *   (arrays of n entries; h_eq may be NULL, or an array whose entries may be
 *   NULL).  Either every frame is queued (tickets[i] for frame i) or, on
 *   INVALID_ARG for any entry or CAPACITY for their total, none is.
 * lsas_server_wait_many: waits up to timeout_ms in total for all n tickets.
 *   On LSAS_ERR_TIMEOUT every ticket stays valid.  Otherwise all n are
 *   consumed; latency_us[i] and status[i] (both nullable arrays) receive each
 *   frame's latency and status, and the call returns the first frame status
 *   that is not LSAS_OK (or LSAS_OK).  INVALID_ARG for an unknown ticket
 *   (nothing consumed).
 * lsas_server_stats: out[0] launches, out[1] frames, out[2] bytes admitted,
 *   out[3] configurations.
 * lsas_server_destroy: finish queued frames, stop the worker, free all; it
 *   returns a device-side condition latched by any configuration's plan
 *   (LSAS_ERR_DEVICE, LSAS_ERR_TIMEOUT) or LSAS_OK.
 * A frame's results do not depend on the other frames it is batched with.
 */
typedef struct lsas_server_s* lsas_server;
lsas_status lsas_server_create(size_t mem_budget_bytes, int max_batch, double max_wait_us,
                               lsas_server* out);
lsas_status lsas_server_register(lsas_server server, int M, int N, int cp_len, int n_sym,
                                 int pilot_idx, int qam_order, lsas_input_fmt fmt,
                                 const float* host_pilot_iq, int* config_id);
lsas_status lsas_server_register_refined(lsas_server server, int M, int N, int cp_len, int n_sym,
                                         int pilot_idx, int qam_order, lsas_input_fmt fmt,
                                         const float* host_pilot_iq,
                                         const uint16_t* d_params_bf16, int* config_id);
lsas_status lsas_server_set_admission(lsas_server server, size_t frame_budget_bytes,
                                      double wait_ms);
lsas_status lsas_server_frame_bytes(lsas_server server, uint64_t out[2]);
lsas_status lsas_server_submit(lsas_server server, int config_id, const void* h_in,
                               float* h_H, uint8_t* h_bits, float* h_eq, uint64_t* ticket);
lsas_status lsas_server_wait(lsas_server server, uint64_t ticket, double timeout_ms,
                             double* latency_us);
lsas_status lsas_server_submit_many(lsas_server server, int n, const int* config_ids,
                                    const void* const* h_in, float* const* h_H,
                                    uint8_t* const* h_bits, float* const* h_eq,
                                    uint64_t* tickets);
lsas_status lsas_server_wait_many(lsas_server server, int n, const uint64_t* tickets,
                                  double timeout_ms, double* latency_us, lsas_status* status);
lsas_status lsas_server_stats(lsas_server server, uint64_t out[4]);
lsas_status lsas_server_destroy(lsas_server server);

/*
 * Learned refinement of the LS channel estimate (Sec. II-C's LS estimate is
 * its input and remains the fallback).  Rows are antenna rows of N
 * subcarriers (R = F*M for a [F][M][N] H); N a multiple of 128 in
 * [128, 2048].  Per row: normalise by the RMS of the row, a residual 1-D
 * convolutional network over subcarriers (2 -> 32 -> 32 -> 32 -> 2
 * channels, kernel 5, ReLU), denormalise.  Parameters: one float vector of
 * LSAS_DN_PARAMS values, W1[32][2][5] b1[32] W2[32][32][5] b2[32]
 * W3[32][32][5] b3[32] W4[2][32][5] b4[2]; the bf16 form has the same order.
 * d_work: caller-owned device scratch of lsas_dn_work_size floats, 16-byte
 *   aligned (INVALID_ARG otherwise).
 *   lsas_dn_apply  d_H [R][N] complex -> d_Hout [R][N] complex (may not
 *                  alias d_H); bf16 != 0 reads bf16 parameters; fp32 sums.
 *   lsas_dn_grad   mean squared error between the network output and the
 *                  true rows d_Htrue normalised by the same RMS -> d_loss[0]
 *                  and the gradient d_grad [LSAS_DN_PARAMS].
 *   lsas_dn_adam   one Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step
 *                  counted from 1) on parameters, first and second moments.
 *   lsas_dn_to_bf16  round the parameters to bf16 (nearest even).
 *   lsas_dn_apply_tc  as lsas_dn_apply with bf16 parameters, the two
 *                  32 -> 32 layers on the tensor cores: bf16 operands, fp32
 *                  sums, each ReLU output rounded to bf16 (nearest even)
 *                  before the next layer.  d_status: caller-owned device
 *                  int, latched to LSAS_ERR_TIMEOUT (6) if a tensor-core
 *                  completion wait gives up after ~2 s (the rows are then
 *                  invalid); never cleared by the library.
 * Errors: INVALID_ARG for bad sizes or null pointers.  Asynchronous.
 */
#define LSAS_DN_PARAMS 10978
lsas_status lsas_dn_work_size(int R, int N, size_t* floats);
lsas_status lsas_dn_apply(const void* d_params, int bf16, const float* d_H, int R, int N,
                          float* d_work, float* d_Hout, void* stream);
lsas_status lsas_dn_grad(const float* d_params, const float* d_Hls, const float* d_Htrue, int R,
                         int N, float* d_work, float* d_grad, float* d_loss, void* stream);
lsas_status lsas_dn_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int step,
                         float lr, void* stream);
lsas_status lsas_dn_to_bf16(const float* d_params, uint16_t* d_params_bf16, void* stream);
lsas_status lsas_dn_apply_tc(const uint16_t* d_params_bf16, const float* d_H, int R, int N,
                             float* d_work, float* d_Hout, int* d_status, void* stream);
/*
 * lsas_dn_grad in BF16 on the tensor cores: the same loss and gradient,
 * with the fp32 parameters d_params rounded to bf16 for the pass (the
 * caller's Adam step keeps them in fp32).  Forward: the tensor-core
 * inference network, storing each ReLU output in bf16 as the next layer
 * reads it.  Backward: the data gradients as tensor-core convolutions with
 * transposed, flipped weights masked by the stored ReLU outputs (bf16), the
 * weight gradients of the two 32 -> 32 layers as tensor-core reductions over
 * positions, those of the two-channel layers and the biases on the CUDA
 * cores; every sum fp32, every reduction in a fixed order.  d_status as
 * lsas_dn_apply_tc.  Errors as lsas_dn_grad (d_work 16-byte aligned).
 */
lsas_status lsas_dn_grad_tc(const float* d_params, const float* d_Hls, const float* d_Htrue,
                            int R, int N, float* d_work, float* d_grad, float* d_loss,
                            int* d_status, void* stream);

/*
 * The learned form of the receiver with the refinement fused after LS
 * (Sec. II-C's LS estimate is its input): per antenna row, the pilot
 * symbol's FFT, LS and the row normalisation feed the tensor-core refinement
 * (as lsas_dn_apply_tc, bf16 parameters d_params_bf16) on chip, so the
 * unrefined estimate is never written to memory; then MRC and demapping
 * with the refined channel (as lsas_demodulate).  Outputs as lsas_run_frame:
 * d_H receives the refined channel.  d_work: lsas_dn_work_size(n_frames * M,
 * N) floats, 16-byte aligned; d_status as lsas_dn_apply_tc.  The plan's
 * other device conditions latch as usual (lsas_plan_sync).
 * Supported: N = 1024 with sc16 input (UNSUPPORTED otherwise); INVALID_ARG
 * for null or misaligned pointers, CAPACITY for n_frames > max_frames.
 * Asynchronous.
 */
lsas_status lsas_run_frame_refined(lsas_plan plan, const void* d_in, int n_frames,
                                   const uint16_t* d_params_bf16, float* d_work, float* d_H,
                                   uint8_t* d_bits, float* d_eq, int* d_status, void* stream);

/*
 * Test hook of failure detection (no counterpart in the paper).  Every wait
 * of the fused kernel on a staging copy is bounded (~2 s, %globaltimer):
 * when it runs out the block latches LSAS_ERR_TIMEOUT, stops issuing
 * copies, skips its remaining waits and finishes.  kind = 1 makes that
 * happen without any fault: block 0's first staging phase also waits for 16
 * bytes that no copy delivers.  kind = 0 (the default) turns it off.
 * Applies to every fused kernel: the per-warp kernel (N <= 1024), the
 * warp-pair kernel (N = 2048, sc16 input) and the warp-specialised kernel
 * (N = 2048, fc32 input).  INVALID_ARG for other kinds.
 */
lsas_status lsas_plan_set_fault(lsas_plan plan, int kind);

/*
 * enable = 1 (the default): lsas_run_frame may split the frames after a
 * batch's last whole wave into antenna shards (see lsas_run_frame), with the
 * shard count chosen for the number of those frames; 2: the same with one
 * shard count for every batch (the single frame's choice, limited so that
 * max_frames frames fit the scratch), so that a frame's results do not
 * depend on how many frames share its call when batches are smaller than
 * one wave (the serving loop uses this); 0: every frame runs unsplit.
 * INVALID_ARG for other values.  Takes effect from the next call.
 */
lsas_status lsas_plan_set_batch_split(lsas_plan plan, int enable);

/*
 * The antenna shards lsas_run_frame would use for the frames after the last
 * whole wave of an n_frames batch (1: no split), into *out_shards.  The
 * choice depends on the plan's shape, the SM count and the batch split
 * setting only.  INVALID_ARG for null pointers or n_frames < 0.
 */
lsas_status lsas_plan_batch_split_shards(lsas_plan plan, int n_frames, int* out_shards);

/*
 * Size of the library's fixed device scratch used by
 * lsas_run_frame_split_static (16 MiB per device).
 */
#define LSAS_STATIC_SCRATCH_BYTES (16u << 20)

/*
 * The antenna-split receiver in one call that allocates no memory.  The
 * paper has no counterpart: this is a library service, not a step of the
 * method.  It computes what lsas_mrc_partial over n_shards even shards (shard
 * g: M / n_shards antennas, one more for the first M % n_shards) followed by
 * lsas_mrc_combine computes, with the shards' partial sums kept in a fixed
 * device array of LSAS_STATIC_SCRATCH_BYTES inside the library instead of in
 * caller buffers.  It is for callers that cannot allocate device memory at
 * call time, for example a receive loop with a per-frame deadline, where
 * cudaMalloc/cudaFree (or a framework allocator growing its pool) would
 * synchronise the device and stall the other streams, or a process whose
 * device memory is fully reserved up front.  It makes no cudaMalloc,
 * cudaFree or other allocating call.
 *   d_in, d_H, d_bits, d_eq: as lsas_run_frame (d_eq may be NULL).
 *   Scratch needed: n_shards * n_frames * (D*N*8 + N*4) bytes; more than
 *   LSAS_STATIC_SCRATCH_BYTES returns LSAS_ERR_CAPACITY before any launch
 *   (for example at M = 64, N = 1024, 13 data symbols: n_shards * n_frames
 *   <= 151).
 * Nothing in the scratch needs to start at zero: the shard pass writes every
 * partial sum that the combine pass of the same call reads.
 * Launches: when n_shards divides M, the shard pass is one launch whose
 * grid row g processes shard g of every frame, so a frame's shards run on
 * different SMs at the same time; for N <= 1024 and small batches
 * (2 * n_frames * n_shards <= SMs) its grid layers also split the data
 * symbols into their groups, each block repeating the pilot transform.
 * Otherwise there is one launch per shard.  Every form gives the same
 * partial sums, hence the same results.
 * The scratch address is looked up (cudaGetSymbolAddress) by
 * lsas_plan_create, with the plan's device current, and kept in the plan, so
 * loading the library's device code and committing the array happen when
 * the plan is made, and no call of this entry point does either.  After a
 * cudaDeviceReset every plan made before it is invalid (its tables and its
 * cached scratch address belong to the destroyed context): make new plans.
 * The scratch is shared by all plans and streams of a device: calls whose
 * execution overlaps on one device race on it and give wrong results, so
 * serialise them (one stream, or synchronise between calls).
 * Errors: INVALID_ARG for a null plan or pointer, n_shards outside [1, M],
 * n_frames < 0 or a d_eq that is not 8-byte aligned (all checked before any
 * launch); CAPACITY as above or for n_frames > max_frames; CUDA if a launch
 * fails.  Asynchronous.
 */
lsas_status lsas_run_frame_split_static(lsas_plan plan, const void* d_in,
                                        int n_frames, int n_shards,
                                        float* d_H, uint8_t* d_bits,
                                        float* d_eq, void* stream);

/*
 * lsas_run_frame on HOST buffers: copies the input to the device, runs the
 * receiver and copies H, bits and (if h_eq is not NULL) eq back, in chunks so
 * that transfers overlap the kernels.  Host buffers should be page-locked
 * (cudaHostAlloc / pinned) for full speed.  The first call on a plan
 * allocates the plan's device staging buffers.  Returns after the results
 * are in host memory (it synchronises stream).  When CP > 0 and a row of N
 * samples spans at least 1 KB, only the N samples after each cyclic prefix
 * cross the host link (the receiver never reads the prefixes): M*S*N*bps
 * bytes per frame instead of M*S*(N+CP)*bps, bps = 4 (SC16) or 8 (FC32).
 */
lsas_status lsas_run_frame_host(lsas_plan plan, const void* h_in,
                                int n_frames, float* h_H, uint8_t* h_bits,
                                float* h_eq, void* stream);

/*
 * Call timing (the paper times each receiver function and averages it;
 * Sec. III).  While a plan's profiling is on, every call of a device entry
 * point on that plan records a CUDA event before and after what it enqueues
 * on its stream; lsas_run_frame_host, which synchronises, is timed on the
 * host clock.  A call that calls another entry point (the per-shard form of
 * lsas_run_frame_split_static) records both.  Profiling is on from creation
 * when the environment variable LSAS_PROFILE is "1", and otherwise follows
 * lsas_plan_set_profile.
 * lsas_plan_profile: waits for the recorded calls to finish, adds them to
 *   per-function totals and writes them as one JSON object,
 *   {"lsas_run_frame": {"calls": 3, "ms": 5.71}, ...}, NUL-terminated, into
 *   buf (len bytes).  needed (nullable) receives the bytes required.  With
 *   buf NULL only the size is reported and nothing is cleared; a successful
 *   write clears the totals.  CAPACITY if len is too small (the totals are
 *   kept), INVALID_ARG for a null plan or both buf and needed null.
 */
lsas_status lsas_plan_set_profile(lsas_plan plan, int on);
lsas_status lsas_plan_profile(lsas_plan plan, char* buf, size_t len, size_t* needed);

/*
 * Synchronise stream, then return and clear the plan's latched device status
 * (LSAS_OK, LSAS_ERR_TIMEOUT or LSAS_ERR_DEVICE), or LSAS_ERR_CUDA.
 */
lsas_status lsas_plan_sync(lsas_plan plan, void* stream);

/*
 * Launch geometry of the plan, for tests and reports: out[0] antennas per
 * step, out[1] threads per block of the fused kernel, out[2] its dynamic
 * shared memory bytes, out[3] data-symbol groups per frame, out[4] staging
 * slots, out[5] 1 if input is staged by bulk asynchronous copies (TMA),
 * out[6] input format, out[7] max_frames.
 */
lsas_status lsas_plan_info(lsas_plan plan, int out[8]);

/*
 * Device memory the plan allocated when it was created, in bytes, into
 * *out_bytes: its tables and the partial-sum scratch of split batch tails
 * (lsas_run_frame).  Buffers made later by the host-buffer entry point or
 * by packet detection are not included.  INVALID_ARG for null pointers.
 */
lsas_status lsas_plan_device_bytes(lsas_plan plan, size_t* out_bytes);

/* Release the plan's device memory (synchronises its device first). */
lsas_status lsas_plan_destroy(lsas_plan plan);

/*
 * Measurement helper, not a step of the method (the paper has no
 * counterpart): the CUDA cores' FP32 FMA throughput on this GPU, against
 * which the FFT's arithmetic rate is reported (an ALU roofline).  Launches
 * blocks x threads threads, each running 8 independent chains of iters packed
 * (f32x2) fused multiply-adds, and writes one float per thread to d_out
 * (blocks * threads floats, caller-owned device memory).  *flops (nullable)
 * receives the FP32 flop count of the launch (an FMA counts 2), which the
 * caller divides by its own CUDA-event time of the launch.  threads must be a
 * multiple of 32 in [32, 512].  INVALID_ARG for bad sizes or a null d_out,
 * CUDA if the launch fails.  Asynchronous on stream.
 */
lsas_status lsas_fma_peak_run(int blocks, int threads, int iters, float* d_out,
                              double* flops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LSAS_H_ */
