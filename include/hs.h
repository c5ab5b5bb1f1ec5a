/*
 * hs.h -- C ABI of libhs.so: the incoherent harmonic sum on one GB300 (sm_103a).
 *
 * Method: Adamek, Roy & Armour, "A Novel Greedy Approach To Harmonic Summing Using GPUs"
 * (arXiv:2202.12817).  For every fundamental bin n of a power spectrum x (1D) or every
 * fundamental (f, z) of an f-fdot plane (2D) the library forms the partial sums of the
 * harmonic orders h = 1..H, normalises each to an SNR with the caller's mean and standard
 * deviation of an h-term sum (Eq. 2), and reports the maximum SNR, the h that reached it and,
 * for the greedy form, the drift path.
 *
 *   simple form (Eq. 3):   S_h[n] = sum_{k=1..h} x[k n]
 *   greedy form (Eq. 5, Algorithm 2): d = 0; at order 1 (with scalloping-loss mitigation,
 *       the default) compare x[n], x[n+1]; at order h >= 2 compare x[m], x[m+1] with
 *       m = h n + d; if the second is strictly larger, d += 1 and it is summed, else the
 *       first is summed.  Path bit h-1 records the increment at order h.
 *   2D greedy: centre (h f + df, h z + dz), best of the 3x3 neighbourhood (centre first, then
 *       raster order dz = -1..1, df = -1..1, strictly larger replaces), 4-bit code
 *       (oz+1)*3 + (of+1) per order at bits 4(h-1)..4h-1.
 *   SNR_h = (S_h - mu[h-1]) / sigma[h-1]; the maximum over h starts at h = 1 and is replaced
 *       only by a strictly larger value (lowest h wins ties).
 *
 * Fundamental domain: 1D n in [0, N_f) with N_f = floor((N-1)/H) -- every read of every form
 * (largest: H n + H) lies inside the spectrum; with HS_FLAG_TRUNCATE_TAIL, n in [0, N - 1), the
 * fundamentals past N_f summing fewer orders.  2D: f in [1, (n_freq-1-H)/H] and the z for which
 * rows z0_row + h z +- h stay inside the plane for all h (see hs_plan_domain_2d).
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA device addresses on the plan's device; the caller owns and
 *     allocates every device buffer.  Device pointers must be 16-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - hs_run and hs_backward never allocate and never synchronise the host.
 *   - Errors are returned as hs_status; nothing throws or aborts across the ABI.  Errors that
 *     only a kernel can see (HS_FLAG_CHECKED) set the plan's device error word, read and
 *     cleared by hs_check_device_error.
 */
#ifndef HS_H
#define HS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HS_OK = 0,
    HS_ERR_INVALID_ARG = 1,    /* a null/misaligned pointer, out-of-range size or flag */
    HS_ERR_UNSUPPORTED = 2,    /* valid but not provided (e.g. a 2D simple form) */
    HS_ERR_OOM = 3,            /* plan-owned device/host allocation failed (plan creation only) */
    HS_ERR_CUDA = 4,           /* a CUDA runtime call failed; see hs_last_cuda_error */
    HS_ERR_DEVICE_BOUNDS = 5,  /* a checked kernel saw an index outside its buffer */
    HS_ERR_DEVICE_TIMEOUT = 6, /* a bounded device wait gave up */
    HS_ERR_NO_DEVICE = 7       /* plan made with HS_FLAG_NO_DEVICE cannot run */
} hs_status;

/* Forms (a bitmask in hs_desc.forms).  HS_FORM_OPTIMAL (1D) is the optimum over every monotone
 * drift path, S*_h[n] = max over D_1..D_h (D_k - D_{k-1} in {0, 1}, D_0 = 0, D_1 = 0 without
 * mitigation) of sum_{k<=h} x[k n + D_k]: the "optimal partial sum" that the greedy choice
 * approximates (Sec. 2.2, Sec. 3), an upper bound on the greedy sum.  It is computed by
 * hs_run_optimal; hs_run computes the simple and greedy forms. */
enum { HS_FORM_SIMPLE = 1, HS_FORM_GREEDY = 2, HS_FORM_OPTIMAL = 4 };

typedef enum { HS_F32 = 0, HS_F16 = 1, HS_BF16 = 2 } hs_dtype;

enum {
    HS_FLAG_NO_MITIGATION = 1u << 0,     /* greedy order 1 sums x[n] without comparing x[n+1] */
    HS_FLAG_PER_SPECTRUM_NORM = 1u << 1, /* mu/sigma are [B][H] instead of [H] */
    HS_FLAG_WHITENING = 1u << 2,         /* load x = fl32(w[j] * p[j]); all lengths equal */
    HS_FLAG_AUTOTUNE = 1u << 3,          /* time candidate launch shapes at plan creation */
    HS_FLAG_GRAPH = 1u << 4,             /* hs_run replays a captured CUDA graph */
    HS_FLAG_NO_DEVICE = 1u << 5,         /* host-only dry run: validate and size, no CUDA calls */
    HS_FLAG_CHECKED = 1u << 6,           /* kernels range-check every index into the error word */
    HS_FLAG_TRUNCATE_TAIL = 1u << 7      /* 1D: also the fundamentals N_f <= n < N - 1, each form with
                                            the orders whose every read fits: simple h n <= N - 1,
                                            greedy / optimal h n + h <= N - 1 (best h <= that count) */
};

/* Plan description. */
typedef struct {
    int32_t dims;            /* 1 (power spectra) or 2 (f-fdot plane) */
    int32_t H;               /* harmonics summed: 1..32 (1D), 1..8 (2D) */
    int32_t forms;           /* any of HS_FORM_SIMPLE | HS_FORM_GREEDY | HS_FORM_OPTIMAL (2D:
                                HS_FORM_GREEDY only) */
    int32_t dtype;           /* hs_dtype of the stored input (spectra or plane); FP32 accumulation */
    int64_t num_spectra;     /* B >= 1 (1D); 1 for 2D */
    const int64_t *lengths;  /* host [B]: N_s bins of spectrum s, H + 1 <= N_s < 2^31 - 64 (1D) */
    const int64_t *offsets;  /* host [B] or NULL: element offset of spectrum s in the concatenated
                                input, each a multiple of 16 bytes / element size; NULL = packed in
                                order, each start rounded up to 32 elements */
    int64_t n_freq;          /* 2D: bins per row (f contiguous) */
    int64_t n_rows;          /* 2D: fdot rows (row-major plane [n_rows][n_freq]) */
    int64_t z0_row;          /* 2D: row holding z = 0 */
    uint32_t flags;          /* HS_FLAG_* */
} hs_desc;

typedef struct hs_plan_s *hs_plan;

/* Per-form inputs and outputs (all device pointers).  F = total fundamentals of the plan
 * (sum over spectra of N_f, concatenated in spectrum order; 2D: z-major, f fastest). */
typedef struct {
    const float *mu;     /* [H] (or [B][H]): mean of an h-term partial sum, entry h-1 (Eq. 2) */
    const float *sigma;  /* same shape: its standard deviation, > 0 */
    float *snr;          /* [F] out: max over h of (S_h - mu) / sigma */
    uint8_t *best_h;     /* [F] out: the h (1..H) of that maximum */
    void *path;          /* [F] out or NULL (greedy only): drift path, uint8/16/32 for H <= 8/16/32;
                            2D: uint32, 4 bits per order */
    uint64_t *argmax;    /* [B] out or NULL: per-spectrum maximum as a key
                            (ordered-float(snr) << 32) | (0xffffffff - n), n the fundamental
                            within the spectrum (2D: the flattened output index); ties -> lowest n */
} hs_form_io;

/* Launch shape of the 1D forward; hs_plan_create picks one (autotuned with HS_FLAG_AUTOTUNE).
 *   kernel 0: one thread per fundamental, read-only gathers of each order's bins;
 *   kernel 1: as 0, the greedy candidates of four orders loaded at once (shorter load chain);
 *   kernel 2: per tile of `threads` fundamentals, each order's window [h n0, h (n0+T-1) + h] is
 *             staged in shared memory by one bulk copy (TMA) into a ring of `stages` slots of
 *             `stage_kb` KiB; `producers` warps issue the copies (copies of one warp complete in
 *             order, so several producer warps keep several in flight), `threads` consumer
 *             threads run both forms from shared memory (not available with HS_FLAG_WHITENING);
 *   kernel 3: as 0 with two fundamentals per thread (n0 + t and n0 + t + threads), their
 *             chains interleaved: half the threads, twice the loads in flight per thread;
 *   kernels 4, 5: as 1 with look-ahead over 2 or 3 orders;
 *   kernel 6: paired lanes: with both forms, two adjacent lanes compute the simple and the greedy
 *             form of one fundamental and issue their reads in the same load instruction (a
 *             tile is threads / 2 fundamentals; with one form, threads fundamentals);
 *   kernel 7: as 6 with two fundamentals per lane (a tile is twice as large). */
typedef struct {
    int32_t kernel;          /* 0..7 */
    int32_t threads;         /* threads per CTA (kernel 2: consumer threads), multiple of 32: 64..256
                                (kernels 0/1/3), 64..512 (kernel 2) */
    int32_t fund_per_thread; /* 2 for kernel 3, else 1 (a tile is threads x fund_per_thread) */
    int32_t ctas_per_sm;     /* persistent grid = ctas_per_sm x SMs; 0 = kernel 0/1: one CTA per
                                tile, kernel 2: as many CTAs as fit on an SM */
    int32_t dynamic;         /* kernels 0/1 with a persistent grid: tiles from an atomic counter in
                                the workspace */
    int32_t stages;          /* kernel 2: ring slots, 2..16 */
    int32_t stage_kb;        /* kernel 2: KiB per slot (>= the largest order window) */
    int32_t prefetch;        /* bit 0 (kernels 2, 6, 7): prefetch the whole input into L2 at launch
                                when it fits in a quarter (kernel 2) or half (6, 7) of L2;
                                bit 1 (all kernels but 2): the tiles of spectrum s prefetch the input
                                of spectrum s+1 into L2, one share each */
    int32_t producers;       /* kernel 2: producer warps, 1..8 (<= stages; threads + 32 producers
                                <= 640) */
} hs_tuning;

/* Create a plan: validates `desc`, computes fundamental counts and tiles, allocates the plan's
 * small device tables and error word on `device`.  *out is NULL on failure. */
hs_status hs_plan_create(hs_plan *out, const hs_desc *desc, int device);
hs_status hs_plan_destroy(hs_plan plan);

/* Fundamental counts per spectrum ([B], host, or NULL) and output offsets ([B+1], host, or NULL). */
hs_status hs_plan_fundamentals(hs_plan plan, int64_t *counts, int64_t *offsets);
/* Element offset of each spectrum in the input ([B+1], host; last = total extent). */
hs_status hs_plan_input_offsets(hs_plan plan, int64_t *offsets);
/* 2D fundamental domain: f in [f_lo, f_hi], z in [z_lo, z_hi]. */
hs_status hs_plan_domain_2d(hs_plan plan, int64_t *f_lo, int64_t *f_hi, int64_t *z_lo, int64_t *z_hi);
/* Bytes of device workspace hs_run / hs_backward take (0 = pass NULL): the forward's dynamic
 * schedule needs 256 bytes; a 1D plan with HS_FLAG_WHITENING adds 4 bytes per input element (hs_run
 * given a workspace first writes the whitened input fl32(w[j] p[j]) there, then runs the pass on
 * that FP32 copy -- the same outputs bit for bit, one gather per loaded value instead of two;
 * without a workspace, and in hs_run_host and hs_run_fixed_scratch, the pass multiplies as it
 * loads); a 2D plane that admits the column sweep (kernel 2 below) adds 16
 * bytes of chain state per fundamental it sweeps and 4 bytes per band; the adjoint uses one
 * partial dL/dw (N floats) per group of spectra (up to 16 groups; required for a whitening plan
 * with grad_w) followed by one byte per (spectrum, 1024-bin block) that marks the blocks
 * receiving contributions. */
hs_status hs_plan_workspace(hs_plan plan, size_t *bytes);
/* Launch shape of the forward.  2D plans take kernel 0 (one thread per (f, z) chain, CTAs over
 * f-tiles fastest) or 1 (the same over z rows fastest, the default: neighbouring z, whose low
 * orders read overlapping rows, stay co-resident), with threads = 256 and every other field 0;
 * or kernel 2, the column sweep: the plane is processed in bands of anchor columns h f, each
 * band's columns of every reachable row staged in shared memory once by a 2D tensor copy and
 * all orders of all chains anchored there run from it, the chain state waiting in the workspace
 * between orders (plane DRAM reads about 2.4x lower than kernel 1 on a 201 x 2^21 plane).
 * Kernel 2 takes threads 256, 512 or 1024 (two warps of which control and publish), stage_kb =
 * band width / 16 (0: 112 columns for FP32, 176 for 16-bit storage, or the widest narrower
 * multiple of 16 the plane takes), stages = 2..4 buffers of one band's tile each (0: 2),
 * ctas_per_sm 0..4, producers 0..64 (chains f < 64 max(1, producers) band widths run whole in
 * registers before the sweep takes over; 0: 64 band widths); it needs rows whose byte stride is
 * a multiple of 16, at most 256 reachable rows, no HS_FLAG_CHECKED, and the workspace (without
 * one, hs_run and hs_run_fixed_scratch run it as kernel 1, with the same outputs bit for bit).
 * The default is kernel 1, except for FP32 planes of 8 or more times the device's L2 size with
 * H >= 6 that the sweep takes: kernel 2 with 1024 threads and producers 5. */
hs_status hs_plan_get_tuning(hs_plan plan, hs_tuning *t);
hs_status hs_plan_set_tuning(hs_plan plan, const hs_tuning *t);

/* Forward pass.  spectra: device input of the plan's dtype at the plan's offsets (2D: the plane).
 * w: device [N] float whitening weights (HS_FLAG_WHITENING) or NULL.  simple / greedy: the
 * forms' I/O (NULL for a form not in the plan).  workspace: >= hs_plan_workspace bytes or NULL
 * when that is 0.  Enqueues on `stream`; graph-capturable.  A 1D pass first clears the argmax keys
 * (and the dynamic schedule's counter) with a small kernel that the pass overlaps (programmatic
 * dependent launch); a whitening plan given a workspace first writes its whitened copy there
 * (which also clears them); a 2D pass clears its key with a stream-ordered memset.  Calls on one
 * plan that share a workspace must not overlap on the GPU. */
hs_status hs_run(hs_plan plan, const void *spectra, const float *w, const hs_form_io *simple,
                 const hs_form_io *greedy, void *workspace, void *stream);

/* Forward pass from host memory, the same results as hs_run.  host_spectra: the input in the
 * plan's layout (hs_plan_input_offsets, extent elements), in page-locked host memory; spectra:
 * a device buffer of extent elements that receives it (16-byte aligned, distinct from
 * host_spectra).  The input is copied in chunks on a stream owned by the plan, and each chunk's
 * fundamentals run on `stream` as soon as the bins they read have arrived (fundamental n reads
 * up to bin H n + H): one spectrum is cut into ranges of fundamentals, a batch into groups of
 * whole spectra (hs_plan_set_host_chunks; one chunk when the spectra do not lie in increasing
 * order, and for 2D plans).  simple / greedy: device outputs as for hs_run.
 * host_simple / host_greedy: NULL, or page-locked host copies of the same outputs (mu and sigma
 * unused; a NULL field is not copied); each chunk's outputs are copied back on a second plan
 * stream while later chunks run (after the whole pass with HS_FLAG_TRUNCATE_TAIL, whose tail
 * needs the whole input), the argmax after the last chunk.  Ordered on `stream`: the copies
 * wait for work already enqueued there, and work enqueued after the call sees the outputs and
 * the host copies.  The first call creates the plan's two copy streams and their events; after
 * that no allocation and no synchronisation, so later calls can be captured in a CUDA graph (each
 * replay copies the buffers' current contents).  Calls on one plan must not overlap on the host. */
hs_status hs_run_host(hs_plan plan, const void *host_spectra, void *spectra, const float *w,
                      const hs_form_io *simple, const hs_form_io *greedy, const hs_form_io *host_simple,
                      const hs_form_io *host_greedy, void *workspace, void *stream);
/* Chunks of hs_run_host's pipeline: 1..16, or 0 for the default (about 16 MiB of input per chunk,
 * at most 8).  One spectrum is cut into chunks of decreasing size (K : K-1 : ... : 1 of its
 * fundamentals), so the pass and output copies that follow the last input copy are short; a
 * batch is cut between spectra, so it may get fewer chunks than asked for. */
hs_status hs_plan_set_host_chunks(hs_plan plan, int32_t chunks);

/* Forward pass of the optimal form (plan with HS_FORM_OPTIMAL, 1D): for every fundamental,
 * the SNR of S*_h (Eq. 2 with the caller's mu/sigma of the optimum), its maximum over h (first
 * strictly larger wins, as for the other forms), the best h and, if optimal->path is set, an
 * optimal drift path of that order (bit k-1 = increment at order k; ties keep the drift, and
 * among the final drifts whose SNR equals the maximum the lowest is taken).  FP32 accumulation
 * along each path.
 * Computed by a dynamic programme over the drift, one warp per fundamental.  Same input and
 * workspace-free; enqueued on `stream` without allocation or synchronisation. */
hs_status hs_run_optimal(hs_plan plan, const void *spectra, const float *w, const hs_form_io *optimal,
                         void *stream);

/* Adjoint of one 1D form with the forward's path and best_h held fixed (a subgradient
 * through the maximum of Eq. 2):
 *   dL/dx[j] = sum over (n, k <= h*(n)) with b_k(n) = j of grad_snr[n] / sigma[h*(n)-1],
 *   b_k(n) = k n (simple) or k n + popcount(path[n] & ((1 << k) - 1)) (greedy, optimal).
 * Each contribution is grad_snr[n] * fl(1/sigma); contributions to each bin are added exactly
 * in 64-bit fixed point (resolution 2^-55 of the largest contribution in its 1024-bin block) and
 * rounded once to FP32 (a result below FP32's normal range may be rounded twice), so the result
 * is bit-reproducible and independent of the order of the additions.
 * grad_in: device [input extent] or NULL: dL/d(spectra); with whitening w[j] dL/dx[j].
 * grad_w: device [N] or NULL (whitening only): dL/dw[j] = sum_s p_s[j] dL/dx_s[j], spectra in
 * order.  fwd: the form's forward outputs (best_h, path, sigma are read).  workspace: >=
 * hs_plan_workspace bytes, or NULL when grad_w is not set.  With a workspace the adjoint first
 * marks the (spectrum, block) pairs that receive a contribution (fundamentals with
 * grad_snr != 0) and skips the candidate search everywhere else, which makes sparse upstream
 * gradients (a top-k loss) cheap; the results are identical either way. */
hs_status hs_backward(hs_plan plan, int32_t form, const float *grad_snr, const hs_form_io *fwd,
                      const void *spectra, const float *w, float *grad_in, float *grad_w,
                      void *workspace, void *stream);

/* Forward pass for callers that cannot allocate device memory (the paper has no counterpart).
 * Same inputs, outputs and results as hs_run, but the scratch hs_run takes as `workspace` (the
 * tile counter of the dynamic schedule) is a fixed 4096-byte array inside the library, held on
 * every GPU that loads the library until the process exits.  Plans needing more workspace than
 * that get HS_ERR_UNSUPPORTED.  Nothing is allocated: no cudaMalloc, cudaFree or allocating
 * library call.  Every call looks up the array's device address with the plan's device current
 * (the address is not cached, so a device reset between calls is harmless); the first call on a
 * device may load the library's device code, so make it before any stream capture.  All calls share the
 * one array and it keeps the last call's contents (the counter is cleared on the stream before
 * every launch), so calls whose work overlaps on the GPU -- on different streams, or of
 * different plans -- race and must be serialised by the caller.  HS_FLAG_GRAPH is ignored here
 * (the work is always launched directly). */
hs_status hs_run_fixed_scratch(hs_plan plan, const void *spectra, const float *w, const hs_form_io *simple,
                               const hs_form_io *greedy, void *stream);

/* Synchronises `stream`, then reads and clears the plan's device error word. */
hs_status hs_check_device_error(hs_plan plan, void *stream);

/* Test of the bounded-wait path: enqueues one CTA that waits on a barrier phase that nothing
 * completes, gives up after limit_us (1..1000000) microseconds and records the timeout in the
 * plan's error word, as the kernels that wait on their own bulk copies do when a wait runs out
 * (kernel 2, 1 s limit).  hs_check_device_error then returns HS_ERR_DEVICE_TIMEOUT; nothing is
 * left in flight and the plan stays usable. */
hs_status hs_selftest_timeout(hs_plan plan, uint32_t limit_us, void *stream);

/* Host helper: closed-form mu/sigma ([H] each, host) of h-term partial sums when every summed
 * term is an independent draw from i.i.d. exponential noise of mean `mean1`: simple h mean1,
 * sqrt(h) mean1; greedy (mitigated) 1.5 h mean1, sqrt(1.25 h) mean1; greedy without mitigation
 * (1 + 1.5 (h-1)) mean1, sqrt(1 + 1.25 (h-1)) mean1; 2D greedy H_9 h mean1,
 * sqrt(h sum_{k<=9} 1/k^2) mean1 (max of 9 draws).  HS_FORM_OPTIMAL has no closed form:
 * HS_ERR_UNSUPPORTED.  No CUDA call. */
hs_status hs_norm_exponential(int32_t form, int32_t dims, int32_t H, int32_t mitigation,
                              double mean1, float *mu_out, float *sigma_out);

const char *hs_status_string(hs_status s);
/* Text of the last CUDA error seen by this thread (empty if none). */
const char *hs_last_cuda_error(void);
/* Library version, e.g. "1.0.0". */
const char *hs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HS_H */
