/*
 * ks.h -- C-ABI of the GB300 (sm_103a) CKKS hybrid KeySwitch library (libks.so).
 *
 * The operation is the KeySwitch of the paper's Sec. II-A / Fig. 1: the input
 * polynomial d at level L (L+1 RNS limbs, NTT form) is split into dnum digits of
 * alpha = ceil((L+1)/dnum) limbs (Table I); each digit is raised to the basis
 * Q u P by iNTT -> fast basis conversion (BConv) -> NTT ("ModUp"), multiplied by
 * its evaluation-key pair and accumulated over the digits; the two accumulated
 * polynomials are then brought back to Q by iNTT -> BConv -> NTT and scaled by
 * P^{-1} ("ModDown"). The four dataflows of Sec. III-A (DigitSerial/DigitParallel
 * x OutputBulk/OutputChunked, Table III) are selectable and compute identical bits.
 *
 * Conventions, all calls:
 *  - Ring Z_q[x]/(x^N + 1), N = 2^log2n. NTT form: slot k holds a(psi^(2 brv(k)+1))
 *    where psi = g^((q-1)/2N) and g is the smallest quadratic non-residue >= 2.
 *  - Polynomials are uint64 limb-major arrays [limb][N]; the Q-limbs come first
 *    (q_0..q_L), then the P-limbs (p_0..p_{alpha-1}); QP = L+1+alpha limbs.
 *  - Digit j covers Q-limbs [j*alpha, min((j+1)*alpha, L+1)); beta =
 *    ceil((L+1)/alpha) digits (beta <= dnum).
 *  - Every residue is canonical ([0, m)) on input and is written canonical.
 *  - "_dev" pointers are device memory (16-byte aligned) owned by the caller;
 *    "_host" pointers are host memory owned by the caller. The library never
 *    frees caller memory.
 *  - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *    stream) unless stated otherwise. Errors found on the host are returned at
 *    once and nothing is launched; CUDA launch errors return KS_ECUDA.
 *  - Return 0 on success or a negative KS_E* code; ks_strerror() names it.
 */
#ifndef KS_H_
#define KS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KS_OK 0
#define KS_EINVAL (-1)    /* bad shape, level, variant, chunks or null pointer */
#define KS_EPRIME (-2)    /* a modulus is not prime, not 1 mod 2N, >= 2^62, or repeated */
#define KS_ENOMEM (-3)    /* device allocation failed */
#define KS_ECUDA (-4)     /* a CUDA call or launch failed */
#define KS_ETIMEOUT (-5)  /* a bounded device-side wait gave up */
#define KS_EALIGN (-6)    /* a pointer is not 16-byte aligned */

/* Dataflows (Sec. III-A, Table III). DS = DigitSerial (digits one after another,
 * one launch sequence per digit), DP = DigitParallel (all digits in one launch),
 * OB = OutputBulk (all output limbs per launch), OC = OutputChunked (the output
 * limbs of each phase split into `chunks` groups processed in turn). */
#define KS_AUTO 0
#define KS_DSOB 1
#define KS_DPOB 2
#define KS_DSOC 3
#define KS_DPOC 4
/* OR-ed into the variant: run BConv, NTT and the key multiply / P^{-1} scaling as
 * separate kernels instead of fusing BConv into the first NTT pass and the
 * element-wise step into the last one (the fusion of Sec. III-B). */
#define KS_UNFUSED 0x100
/* OR-ed into the variant: register rounds of radix 4 (4 points per thread, twice the
 * threads per tile) instead of radix 8; more parallelism for small workloads. */
#define KS_RADIX4 0x200
/* OR-ed into the variant: register rounds of radix 16 (16 points per thread, half the
 * threads per tile): fewer shared-memory round trips for large workloads. */
#define KS_RADIX16 0x400
/* Radix schedule, OR-ed into the variant: the register-round radix of one kernel stage,
 * overriding the plan's for that stage only. Stages: KS_ST_INV (the input iNTT and the
 * iNTT of the accumulators' P-limbs), KS_ST_UPC (ModUp BConv + first NTT pass),
 * KS_ST_KM (second NTT pass + key multiply), KS_ST_DNC (ModDown BConv + first NTT
 * pass), KS_ST_DNR (second NTT pass + P^{-1} scaling). Radix codes: KS_R4, KS_R8,
 * KS_R16. Every schedule computes the same bits. */
#define KS_STAGE_SHIFT 16
#define KS_ST_INV 0
#define KS_ST_UPC 1
#define KS_ST_KM 2
#define KS_ST_DNC 3
#define KS_ST_DNR 4
#define KS_R4 1
#define KS_R8 2
#define KS_R16 3
#define KS_STAGE_RADIX(stage, code) ((code) << (KS_STAGE_SHIFT + 2 * (stage)))
/* OR-ed into the variant: a stage's column pass (N >= 2^13) uses the alternative column
 * tile (2^11 points instead of 2^10 up to N = 2^15, 2^10 instead of 2^11 above): the
 * inverse NTTs (KS_COLALT_INV), the ModUp BConv pass (KS_COLALT_UPC), the ModDown BConv
 * pass (KS_COLALT_DNC), or all three (KS_COLTILE_ALT). */
#define KS_COLALT_INV 0x4000000
#define KS_COLALT_UPC 0x8000000
#define KS_COLALT_DNC 0x10000000
#define KS_COLTILE_ALT (KS_COLALT_INV | KS_COLALT_UPC | KS_COLALT_DNC)
/* OR-ed into a fused DPOB variant at N >= 2^13 (other plans ignore it): the key multiply
 * of the Q-limb targets runs on a second stream of the context while, on `stream`, the
 * P-limb targets' key multiply is followed by the iNTT of the accumulators' P-limbs and
 * the ModDown BConv pass (they need only the P-limb accumulators); the two join before
 * the last ModDown pass. Same result bits; calls on one context serialize this fork. */
#define KS_SPLIT_DOWN 0x20000000
/* OR-ed into a fused variant: the ModUp and ModDown basis conversions (Sec. II-A) run on
 * the tensor cores (tcgen05): both operands split into bytes, exact bf16 x bf16 -> fp32
 * products summed below 2^23, recombined into the exact 128-bit sum and reduced once,
 * fused with the first forward NTT pass (the inverse column passes write the bytes of
 * their output instead of the output). Same result bits as the integer path. Effective
 * on contexts with ks_info.tc = 1 (2^13 <= N <= 2^17, 2 <= alpha <= 9, dnum <= 64); ignored
 * otherwise and by unfused plans. */
#define KS_BCONV_TC 0x800
/* OR-ed into a fused variant: the ModDown basis conversion alone runs on the tensor cores
 * as KS_BCONV_TC describes; the ModUp conversion stays on the integer path. Same
 * conditions as KS_BCONV_TC, which includes it. */
#define KS_BCONV_TC_DOWN 0x1000

typedef struct {
  uint32_t dnum;     /* decomposition number (>= 1) */
  uint32_t log2n;    /* N = 2^log2n, 1 <= log2n <= 17 */
  uint32_t L;        /* level: the input has L+1 limbs (1 <= L+1 <= 128) */
  const uint64_t *q; /* host array of the L+1 ciphertext primes */
  uint32_t nq;       /* must equal L+1 */
  const uint64_t *p; /* host array of the alpha special primes */
  uint32_t np;       /* must equal alpha = ceil((L+1)/dnum) */
} ks_params;

typedef struct {
  uint32_t N, alpha, beta, QP, nq, np;
  size_t evk_words; /* words of the key that a KeySwitch reads: beta*2*QP_top*N, the
                       first beta digit pairs of the top level's key */
  size_t in_words;  /* (L+1)*N */
  size_t out_words; /* 2*(L+1)*N */
  size_t table_bytes; /* device bytes held by the context's constant tables */
  int tuned_variant;  /* plan picked by ks_tune (0 = not tuned) */
  int tuned_chunks;
  int tuned_batch;    /* batch size it was tuned for */
  float tuned_ms;     /* its time per KeySwitch in the tuning run */
  int L;              /* level of this context (nq = L+1) */
  int top_L;          /* level of the context whose keys it reads (= L unless a level view) */
  int selected_variant; /* plan picked by ks_select (0 = none) */
  int selected_chunks;
  int tc;               /* 1: KS_BCONV_TC is effective on this context */
} ks_info;

typedef struct ks_context ks_context;

/* Validates the parameters (primality by deterministic Miller-Rabin, q = 1 mod 2N,
 * q < 2^62, all distinct) and builds the twiddle and basis-conversion tables on
 * the current device (synchronous). On success *out owns them until
 * ks_context_destroy. Returns KS_EINVAL / KS_EPRIME / KS_ENOMEM / KS_ECUDA. */
int ks_context_create(const ks_params *prm, ks_context **out);

/* Frees the context's tables and internal workspace. NULL is ignored. */
void ks_context_destroy(ks_context *ctx);

int ks_context_info(const ks_context *ctx, ks_info *info);

/* A level view of `top` for KeySwitches at level `level` (0 <= level <= top's L):
 * Q = q_0..q_level, the same alpha special primes, digits of alpha limbs
 * (beta = ceil((level+1)/alpha)), and the top level's keys: a KeySwitch on the view
 * reads the first beta digit pairs of a key made for `top`, with its limbs at the
 * top level's positions. The level falls by one per multiplication and the best
 * dataflow changes with it (Sec. II-A on levels; Sec. V on switching the dataflow
 * as L changes within a workload): each view has its own plan and tuner state.
 * The view owns its own tables; `top` may be destroyed first. Key generation on a
 * view returns KS_EINVAL (keys are made at the top level). */
int ks_context_at_level(const ks_context *top, int level, ks_context **out);

/* Evaluation keys from given randomness (the random draws are inputs):
 *   evk_j = (b_j, a_j), b_j = -a_j*s_to + e_j + [P*g_j]*s_from over Q u P,
 * with g_j = 1 mod the primes of digit j, 0 mod every other prime.
 *   s_from_dev [N] int8 ternary: the key switched FROM (s'); s_to_dev [N] int8: TO (s)
 *   a_dev      [beta][QP][N] uint64, uniform, NTT form
 *   e_dev      [beta][N] int32, small error (coefficient form)
 *   evk_dev    [beta][2][QP][N] uint64 output, NTT form (pair index 0 = b, 1 = a)
 * Not on the timed path; allocates and frees its own scratch. */
int ks_keygen(ks_context *ctx, const int8_t *s_from_dev, const int8_t *s_to_dev,
              const uint64_t *a_dev, const int32_t *e_dev, uint64_t *evk_dev,
              void *stream);

/* Relinearisation key for HMUL (Sec. II-A): ks_keygen with s_from = s^2 (the
 * square in the ring, formed on the device) and s_to = s. Same a, e and evk layout. */
int ks_keygen_relin(ks_context *ctx, const int8_t *s_dev, const uint64_t *a_dev,
                    const int32_t *e_dev, uint64_t *evk_dev, void *stream);

/* Rotation key for HROT (Sec. II-A): ks_keygen with s_from = s(x^k), the Galois
 * automorphism of s for the odd element k in [1, 2N) (rotation by r slots:
 * k = 5^r mod 2N; conjugation: k = 2N - 1), and s_to = s. */
int ks_keygen_galois(ks_context *ctx, const int8_t *s_dev, uint32_t galois_elt,
                     const uint64_t *a_dev, const int32_t *e_dev, uint64_t *evk_dev,
                     void *stream);

/* Device bytes of scratch that ks_switch needs for (variant, chunks). */
int ks_workspace_size(const ks_context *ctx, int variant, int chunks, size_t *bytes);

/* One KeySwitch (Sec. II-A, Fig. 1) at level L (at the view's level for a level view,
 * whose evk is the top level's key).
 *   d_dev   [L+1][N]            input, NTT form
 *   evk_dev [beta][2][QP][N]    keys from ks_keygen (or any canonical keys)
 *   out_dev [2][L+1][N]         output pair, NTT form; must not alias the inputs
 *   variant KS_DSOB..KS_DPOC (| KS_UNFUSED | KS_RADIX4 | KS_RADIX16 | a radix schedule
 *           KS_STAGE_RADIX(..) | KS_COLALT_* | KS_SPLIT_DOWN | KS_BCONV_TC |
 *           KS_BCONV_TC_DOWN), or KS_AUTO (the plan ks_tune chose for this context,
 *           else the one ks_select chose, else DPOB fused radix 8; the last two with
 *           KS_BCONV_TC added where ks_info.tc = 1, N >= 2^16 and L+1 > alpha)
 *   chunks  1..64 output groups for the OC variants (0 = 2; the paper searches 2..10);
 *           ignored for OB
 *   workspace_dev / workspace_bytes: caller scratch of at least
 *           ks_workspace_size() bytes, or NULL/0 to use the context's internal
 *           workspace (allocated on first use and grown as needed; calls that use it
 *           must then be ordered, e.g. issued on one stream).
 * Asynchronous on `stream`. The kernels are chained by programmatic dependent launch
 * (consecutive calls on a stream overlap their boundaries); for N <= 2^12 repeated
 * calls with the same plan, buffers and stream replay a cached CUDA graph. */
int ks_switch(ks_context *ctx, const uint64_t *d_dev, const uint64_t *evk_dev,
              uint64_t *out_dev, int variant, int chunks, void *workspace_dev,
              size_t workspace_bytes, void *stream);

/* Operations for ks_eval_workspace_size. */
#define KS_OP_SWITCH 0
#define KS_OP_HMUL 1
#define KS_OP_HROT 2

/* Device bytes of scratch that ks_switch / ks_hmul / ks_hrot need. */
int ks_eval_workspace_size(const ks_context *ctx, int op, int variant, int chunks,
                           size_t *bytes);

/* HMUL (Sec. II-A): for ciphertexts ct1 = (x0, x1), ct2 = (y0, y1) over Q in NTT form,
 *   out = (x0 y0, x0 y1 + x1 y0) + KS(x1 y1)
 * with KS under the relinearisation key rlk (ks_keygen_relin). No rescaling.
 *   ct1_dev, ct2_dev, out_dev  [2][L+1][N] uint64 device, canonical residues;
 *   out may alias ct1 or ct2.  rlk_dev as evk_dev of ks_switch.
 * The tensor product is one element-wise kernel (x1 y1 into the workspace); the
 * final additions are folded into the KeySwitch's last kernel. variant, chunks,
 * ws, ws_bytes and stream as for ks_switch (ws: ks_eval_workspace_size KS_OP_HMUL). */
int ks_hmul(ks_context *ctx, const uint64_t *ct1_dev, const uint64_t *ct2_dev,
            const uint64_t *rlk_dev, uint64_t *out_dev, int variant, int chunks, void *ws,
            size_t ws_bytes, void *stream);

/* HROT (Sec. II-A): rotation of ct = (c0, c1) by the Galois element k,
 *   out = (sigma_k(c0), 0) + KS(sigma_k(c1)),  sigma_k(a)(x) = a(x^k),
 * with KS under the rotation key rtk (ks_keygen_galois with the same k). The
 * paper's formula swaps the roles of c0 and c1 relative to its HMUL; this follows
 * the HMUL's convention (decryption c0 + c1 s). In the NTT domain sigma_k is a
 * permutation of the slots (one gather kernel).
 *   ct_dev, out_dev [2][L+1][N] uint64 device (out may alias ct); k odd in [1, 2N).
 * Other arguments as for ks_hmul (ws: KS_OP_HROT). */
int ks_hrot(ks_context *ctx, const uint64_t *ct_dev, uint32_t galois_elt,
            const uint64_t *rtk_dev, uint64_t *out_dev, int variant, int chunks, void *ws,
            size_t ws_bytes, void *stream);

/* ks_switch with host buffers d_host [L+1][N] and out_host [2][L+1][N]; evk stays
 * device-resident; synchronizes `stream` before returning.
 *   Pinned (page-locked, device-mapped) buffers: the first kernel reads the input
 *   straight from host memory over the CPU-GPU link and the last kernel writes the
 *   result straight into host memory (no staging copies); both must be 16-byte
 *   aligned (else KS_EALIGN).
 *   Pageable buffers: copied through device staging buffers owned by the context.
 * Both host buffers must stay valid and unmodified by other threads until return. */
int ks_switch_host(ks_context *ctx, const uint64_t *d_host, const uint64_t *evk_dev,
                   uint64_t *out_host, int variant, int chunks, void *stream);

/* ks_switch_host without the synchronization, for streams of host-buffer KeySwitches:
 * d_host and out_host must be pinned, device-mapped buffers (cudaHostAlloc /
 * cudaHostRegister; anything else returns KS_EINVAL and launches nothing), 16-byte
 * aligned (else KS_EALIGN). The first kernel reads d_host over the CPU-GPU link and
 * the last one writes out_host; the result is there once `stream` has passed this call
 * (an event or a synchronize), and d_host must stay unmodified until then. Calls on one context share its staging
 * buffer and workspace, so they must be ordered (issued on one stream); consecutive
 * calls are chained like ks_switch's (N <= 2^12: cached graph replay). */
int ks_switch_host_async(ks_context *ctx, const uint64_t *d_host, const uint64_t *evk_dev,
                         uint64_t *out_host, int variant, int chunks, void *stream);

/* Host-buffer KeySwitch on a caller scratch, for host-buffer KeySwitches of one context
 * in flight on several streams at once (each stream with its own scratch): the input is
 * copied to the device and the result back by the copy engines (cudaMemcpyAsync on
 * `stream`), around kernels on device buffers, so one call's transfers overlap another
 * call's kernels. d_host ([L+1][N]) and out_host ([2][L+1][N]) must be pinned,
 * device-mapped host memory (else KS_EINVAL); the result is in out_host once `stream`
 * has passed this call, and d_host must stay unmodified until then. ws: device scratch
 * of ks_host_workspace_size bytes (the workspace, then device copies of the input and
 * of the result), 16-byte aligned, not used by another call in flight; smaller scratch
 * returns KS_EINVAL and queues nothing. No synchronization, no graph cache. */
int ks_host_workspace_size(const ks_context *ctx, int variant, int chunks, size_t *bytes);
int ks_switch_host_async_ws(ks_context *ctx, const uint64_t *d_host, const uint64_t *evk_dev,
                            uint64_t *out_host, int variant, int chunks, void *ws_dev,
                            size_t ws_bytes, void *stream);

/* ks_switch without any device allocation, for callers that cannot allocate device
 * memory when they switch keys: callers held to a fixed allocator or memory-pool
 * budget that forbids new device allocations, and real-time or embedded integrations
 * that must not call the allocator (which can block and synchronize the device) after
 * start-up. The paper has no counterpart; this is a deployment variant of ks_switch
 * (same arguments, same result bits).
 *   Scratch: a static device array of ks_noalloc_scratch_bytes() bytes (128 MiB) in
 *   this library; every GPU that loads it holds it until the process exits. The
 *   caller still passes the inputs and the output.
 *   Limit: if ks_workspace_size(ctx, variant, chunks) exceeds that size, returns
 *   KS_EINVAL and launches nothing (e.g. (4,2^16,35) fits with KS_DSOC and
 *   chunks >= 4, not with KS_DPOB).
 *   Device: the current device must be the context's (else KS_EINVAL).
 *   Set-up: the first call on a device looks up the array's device address (with
 *   that device current) and keeps it for the life of the process. A device reset
 *   (cudaDeviceReset) is not supported.
 *   Sharing: every call uses the same array and leaves its contents behind; no part
 *   of it needs to start at zero. Calls that overlap on the GPU (other streams,
 *   other threads) race on it: order them, e.g. on one stream.
 *   Launches the KeySwitch kernels directly on `stream` at every size (no graph cache
 *   and no context arena), and calls no cudaMalloc, cudaFree or other allocating
 *   routine. */
size_t ks_noalloc_scratch_bytes(void);
int ks_switch_noalloc(ks_context *ctx, const uint64_t *d_dev, const uint64_t *evk_dev,
                      uint64_t *out_dev, int variant, int chunks, void *stream);

/* A batch of independent KeySwitches of uneven (dnum, N, L). */
typedef struct {
  ks_context *ctx;
  const uint64_t *d_dev;   /* [L+1][N] */
  const uint64_t *evk_dev; /* [beta][2][QP][N] */
  uint64_t *out_dev;       /* [2][L+1][N] */
  int variant;             /* dataflow for this job (as in ks_switch); 0 = KS_AUTO */
  int chunks;              /* OutputChunked groups (0 = the context's or 2) */
} ks_job;

#define KS_BATCH_GRAPH 0x1    /* capture the batch in a CUDA graph, replay it on later
                                 calls with the same jobs (same pointers) */
#define KS_BATCH_AUTOTUNE 0x2 /* ks_tune each context first (once per group size) */
#define KS_BATCH_PERSISTENT 0x4 /* run the whole batch in persistent kernels, one per
                                   stage over every job (every job's N in
                                   2^13..2^17; plans DPOB, fused) */
#define KS_BATCH_SELECT 0x8  /* jobs naming KS_AUTO run the plan of the installed selector
                                network (ks_select, run once per context and selector);
                                not with KS_BATCH_AUTOTUNE or KS_BATCH_PERSISTENT */
#define KS_BATCH_TEST_STALL 0x100 /* tests only, with KS_BATCH_PERSISTENT: run the batch
                                     as one dataflow kernel (below) and make one of its
                                     dependencies unreachable, so that the bounded wait
                                     gives up and ks_batch_status reports KS_ETIMEOUT */

/* With KS_BATCH_PERSISTENT, one persistent kernel per stage runs the batch (input
 * iNTT rows, columns, ModUp, key multiply, accumulator iNTT rows, columns, ModDown
 * columns, ModDown rows; the key multiply and ModDown rows in two launches, N >= 2^16
 * and N <= 2^15): each launch's CTAs claim the tiles of that stage of every job, and
 * each launch waits for the previous one (programmatic dependent launch). With KS_BATCH_TEST_STALL the batch runs instead as one dataflow kernel
 * whose tiles wait, with a bounded wait (about 2 s of device time), for the tiles they
 * read; a wait that runs out sets a device error word and every CTA returns;
 * ks_batch_status then reports KS_ETIMEOUT. The persistent grids assume they have the
 * GPU to themselves while they run.
 *
 * Runs njobs independent KeySwitches on `stream` (asynchronous). Jobs sharing a
 * context form a group: its jobs share every kernel launch (up to 16 jobs per
 * launch, grid z) with the job's plan (KS_AUTO: the context's tuned plan, or with
 * KS_BATCH_SELECT the selector's). Groups run concurrently on internal streams
 * forked from and joined back to `stream`. The scratch is a
 * library-owned arena (grown on demand, outside any capture). Calls are serialized
 * internally; the arena is shared, so batches must not overlap on the GPU with other
 * batches (issue them on one stream). With KS_BATCH_GRAPH the whole batch is one
 * CUDA graph launch after the first call. */
int ks_switch_batch(const ks_job *jobs, int njobs, int flags, void *stream);

/* Synchronizes `stream` and reads the error word of the last persistent batch
 * launched by this process: KS_OK, or KS_ETIMEOUT if a bounded wait gave up. */
int ks_batch_status(void *stream);

/* Autotuner: times the dataflows {DPOB, DSOB, DPOC c=2, DPOC c=4, DSOC c=2} x
 * {radix 8, radix 4, radix 16} on this job (replicated `batch` times, 1..16, in one
 * launch set); then, for N >= 2^13, refines the winner's schedule one coordinate at a
 * time: each stage's radix (KS_STAGE_RADIX), each column pass's tile (KS_COLALT_*) and,
 * for DPOB, the split ModDown (KS_SPLIT_DOWN), a change kept when the KeySwitch gets
 * more than 1.5% faster (best of six timings each). Stores the result as the
 * context's KS_AUTO plan and writes it to *variant / *chunks. Writes the switched
 * result to out_dev. Synchronizes `stream`; allocates and frees its own scratch. */
int ks_tune(ks_context *ctx, const uint64_t *d_dev, const uint64_t *evk_dev, uint64_t *out_dev,
            int batch, int *variant, int *chunks, void *stream);

/* Reads and clears the context's sticky device error word (bounded waits that
 * gave up). Synchronizes `stream`. Returns KS_OK or KS_ETIMEOUT. */
int ks_sync_status(ks_context *ctx, void *stream);

/* Dataflow selector: an MLP 6 -> 64 -> 64 -> 4 (ReLU, FP32) that maps workload
 * features to predicted latencies of four candidate plans (the encoding and the
 * features are those of ks_selector below). The paper motivates
 * it (parameter-aware choice of the dataflow, Sec. V) but gives no model; it never
 * touches the KeySwitch arithmetic. Parameters: KS_MLP_PARAMS floats,
 *   W1[6][64] | b1[64] | W2[64][64] | b2[64] | W3[64][4] | b3[4]
 * (W[i][j]: input i to output j). x [batch][6], y / t / mask [batch][4], all device
 * float arrays, batch <= KS_MLP_MAX_BATCH. Asynchronous on `stream`. */
#define KS_MLP_PARAMS 4868
#define KS_MLP_MAX_BATCH 4096
int ks_mlp_forward(const float *params_dev, const float *x_dev, int batch, float *y_dev,
                   void *stream);
/* Gradient of the masked mean-squared loss sum(mask (y - t)^2) / sum(mask) with
 * respect to every parameter (grad_dev: KS_MLP_PARAMS floats), and the loss. */
int ks_mlp_grad(const float *params_dev, const float *x_dev, const float *t_dev,
                const float *mask_dev, int batch, float *grad_dev, float *loss_dev,
                void *stream);
/* `steps` full-batch Adam steps (lr, beta1 0.9, beta2 0.999, eps 1e-8) on params_dev in
 * place; adam_m / adam_v: moment buffers (KS_MLP_PARAMS floats each, zero at the start),
 * step0: steps already taken (bias correction), grad_scratch: KS_MLP_PARAMS floats,
 * loss_dev: `steps` floats, the loss before each update. One launch. */
int ks_mlp_train(float *params_dev, float *adam_m_dev, float *adam_v_dev, float *grad_scratch,
                 const float *x_dev, const float *t_dev, const float *mask_dev, int batch,
                 int steps, float lr, int step0, float *loss_dev, void *stream);

/* The learned dataflow selector inside the library (a parameter-aware choice of the
 * dataflow, as Sec. V proposes): a trained 6-64-64-4 network (KS_MLP_PARAMS floats in
 * the layout of ks_mlp_forward), its standardisation and its four candidate plans.
 *   Features of a context with n_Q = L+1 Q-limbs, alpha special primes, beta digits,
 *   QP = n_Q + alpha and d = dnum (a level view: d = beta), against l2_bytes (0: the
 *   current device's L2 size): log2 N, n_Q, d, log2(beta QP N 8 / l2),
 *   log2(QP N 8 / l2), log2(2 beta QP N 8 / l2) (the DPOB and DSOB ModUp working sets
 *   and the key bytes, Table III); the network sees (f - x_mean) / x_std.
 *   Output k (standardised) decodes as e_k = y_k t_std[k] + t_mean[k]; the predicted
 *   log-latency of candidate 0 is e_0, of candidate k >= 1 e_0 + e_k; the pick is the
 *   smallest (the first on ties). */
typedef struct {
  float params[KS_MLP_PARAMS];
  double x_mean[6], x_std[6];
  double t_mean[4], t_std[4];
  int variant[4], chunks[4]; /* candidate plans (as for ks_switch) */
  long long l2_bytes;
} ks_selector;

/* Installs a copy of `sel` for this process, its parameters on the current device
 * (synchronous). KS_EINVAL for a null pointer, a non-finite value, a standard
 * deviation <= 0, a negative l2_bytes or an invalid plan; KS_ENOMEM / KS_ECUDA. */
int ks_selector_load(const ks_selector *sel);

/* Runs the installed network for `ctx` (one ks_mlp_forward launch on `stream`, which
 * it then synchronizes) and records the pick as the context's selected plan: KS_AUTO
 * uses it when ks_tune has not chosen one, and ks_switch_batch with KS_BATCH_SELECT
 * uses it for jobs naming KS_AUTO. Writes the plan to *variant / *chunks when not
 * null (ks_info.selected_variant reports the same pick). The selected plan runs with
 * KS_BCONV_TC added where the context has the tensor-core path (ks_info.tc), N >= 2^16
 * and the input spans more than one digit (L+1 > alpha). KS_EINVAL when no selector is
 * installed on the current device. */
int ks_select(ks_context *ctx, int *variant, int *chunks, void *stream);

/* Per-kernel timing with CUDA events, for measurement. Between ks_profile_begin and
 * ks_profile_end every kernel launch made by ks_switch on this thread is bracketed
 * by an event pair on its stream and tagged with its algorithmic traffic (the
 * bytes it must read and write at least: each input and output once) and its
 * modular operation count (butterflies, multiply-accumulates, scalings).
 * ks_profile_end synchronizes those events and aggregates them by kernel name. */
typedef struct {
  char name[40];
  int launches;
  double ms;     /* summed event time */
  double bytes;  /* summed algorithmic bytes */
  double ops;    /* summed modular operations */
  double macs;   /* of which exact 128-bit multiply-accumulate terms (basis conversion,
                    key multiply) and Montgomery reductions; the rest are Shoup products
                    (butterflies, scalings) */
  double tensor_flops; /* summed tensor-core FLOPs (2 per bf16 multiply-add), counted
                          apart from ops: the basis conversions of KS_BCONV_TC plans */
} ks_kernel_stat;

int ks_profile_begin(void);
int ks_profile_end(ks_kernel_stat *stats, int max_stats, int *count);

/* Throughput ceiling of the library's modular arithmetic on the current device,
 * measured: one launch of `iters` iterations on every SM at full occupancy, with no
 * memory traffic, timed with CUDA events on `stream` (after one shorter warm-up
 * launch; synchronizes `stream`). It is the measured denominator for kernels bound by
 * the integer pipes, beside the one derived from unit counts and clocks.
 *   KS_CAL_BUTTERFLY: forward lazy butterflies (one approximate-quotient Shoup
 *                     product, an add and a subtract) per second;
 *   KS_CAL_MAC:       exact 64x64->128-bit multiply-accumulate terms per second, one
 *                     Montgomery reduction per 8 terms.
 * *ops_per_s receives the rate. Returns KS_EINVAL (unknown kind, iters < 1, null
 * pointer), KS_ENOMEM or KS_ECUDA. */
#define KS_CAL_BUTTERFLY 1
#define KS_CAL_MAC 2
int ks_calibrate(int kind, int iters, double *ops_per_s, void *stream);

const char *ks_strerror(int code);

/* The CUDA runtime's message for the last CUDA error that made a call of this
 * thread return KS_ECUDA or KS_ENOMEM ("no error" if none). */
const char *ks_cuda_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* KS_H_ */
