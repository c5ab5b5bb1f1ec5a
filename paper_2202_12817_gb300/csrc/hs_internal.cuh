// Internal definitions shared by the harmonic-sum kernels and the plan / C-ABI code.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hs.h"

namespace hs {

constexpr int kMaxH1D = 32;
// adjoint: spectra with at most this many nonzero upstream gradients stage contributions from a
// list of those fundamentals instead of scanning every candidate of a bin block
constexpr int kBwdListCap = 64;
constexpr int kMaxH2D = 8;

// Device error word values (first error wins).
constexpr int kErrNone = 0;
constexpr int kErrBounds = 1;
constexpr int kErrTimeout = 2;

// Per-form arguments of the forward kernels.
struct FormArgs {
    const float *mu;
    const float *sigma;
    float *snr;
    uint8_t *best_h;
    void *path;
    unsigned long long *argmax;
};

// 1D forward launch arguments.
struct Fwd1DArgs {
    const void *x;                 // concatenated spectra (dtype of the plan)
    const float *w;                // whitening weights [N] or nullptr
    const int64_t *in_off;         // [B+1] element offset of each spectrum
    const int64_t *fund_off;       // [B+1] output offset of each spectrum (prefix of its fundamentals)
    const int64_t *nf_main;        // [B] fundamentals with all H orders, N_f = floor((N-1)/H)
    const int64_t *tail_tile_start;// [B+1] prefix of truncated-tail tiles (HS_FLAG_TRUNCATE_TAIL): the
                                   // fundamentals N_f <= n < min(N - 1, n1), n1 = floor((N - 1) / 2) + 1
    int64_t tail_tiles;            // total truncated-tail tiles (0 without the flag)
    const int64_t *tail1_tile_start;// [B+1] prefix of one-order tail tiles: max(n1, N_f) <= n < N - 1,
                                   // where both forms keep order 1 only
    int64_t tail1_tiles;           // total one-order tail tiles
    const int64_t *tile_start;     // [B+1] prefix of tiles per spectrum
    const int64_t *in_len;         // [B] N_s (for checked mode)
    int32_t B;
    uint32_t tiles_per_spec;       // > 0: every spectrum has this many main-pass tiles (one length for
                                   // all, fewer than 2^22 tiles in all)
    uint32_t tail_tiles_per_spec;  // > 0: likewise for the truncated-tail tiles
    uint32_t tail1_tiles_per_spec; // > 0: likewise for the one-order tail tiles
    float inv_tiles_per_spec;      // fl(1 / tiles_per_spec)
    int32_t H;
    int32_t mitigation;
    int32_t per_spectrum_norm;
    int32_t path_bytes;            // 0, 1, 2 or 4
    int32_t checked;
    int32_t fund_per_thread;
    int64_t total_tiles;
    unsigned long long *tile_counter;  // dynamic schedule (nullptr = static)
    int64_t extent;                // readable elements of the input buffer (vector loads stay below)
    int64_t pf_chunk;              // > 0: CTA i first prefetches input bytes [i c, (i+1) c) into L2
    int64_t pf_bytes;              // input bytes covered by that prefetch
    int32_t pf_next;               // 1: the tiles of spectrum s prefetch spectrum s+1 into L2, one share each
    int32_t elem_bytes;            // bytes per stored element
    FormArgs s;                    // simple form outputs (unused unless the form is on)
    FormArgs g;                    // greedy form outputs
    int *err;                      // device error word
};

// Shared-memory staging plan of the window kernel (kernel 2): the (tile, order) sequence of a
// CTA streams through a ring of `nslot` slots of `slot_bytes` each; order j goes to slot
// j % nslot and its bulk copy is issued by producer warp j % nprod.
struct WinPlan {
    int32_t T;                        // fundamentals per tile (= consumer threads)
    int32_t nslot;                    // ring slots (2..16)
    int32_t nprod;                    // producer warps (1..8)
    int32_t slot_bytes;               // bytes per slot (>= the largest order window)
    int64_t extent;                   // readable elements of the input buffer
    int64_t pf_chunk;                 // > 0: CTA i first prefetches input bytes [i c, (i+1) c) into L2
};

// Bytes of the order-h window of a T-fundamental tile: h (T-1) + h + 1 elements plus up to
// one 16-byte alignment unit at each end, rounded to 16 bytes.
inline int64_t win_bytes(int h, int T, int elem)
{
    const int64_t a = 16 / elem;
    const int64_t n = static_cast<int64_t>(h) * (T - 1) + h + 1 + 2 * (a - 1);
    return (n * elem + 15) / 16 * 16;
}

constexpr int kWinStaticSmem = 2048;  // static shared memory of the window kernel (upper bound)

// 2D forward launch arguments.
struct Fwd2DArgs {
    const void *plane;             // [n_rows][n_freq] of the plan's dtype
    int64_t n_freq;
    int64_t n_rows;
    int64_t z0_row;
    int32_t H;
    int64_t f_lo, nff;             // f in [f_lo, f_lo + nff)
    int64_t z_lo, nz;              // z in [z_lo, z_lo + nz)
    int32_t checked;
    int32_t zfast;                 // 1: grid.x runs over z, grid.y over f-tiles
    FormArgs g;
    int *err;
};

// 1D adjoint launch arguments.
struct Bwd1DArgs {
    int32_t form;
    int32_t H;
    int32_t B;
    int32_t path_bytes;
    const float *grad_snr;
    const uint8_t *best_h;
    const void *path;
    const float *sigma;
    int32_t per_spectrum_norm;
    const void *p;                 // spectra (for grad_w / whitening)
    int32_t dtype;
    const float *w;
    const int64_t *in_off;
    const int64_t *in_len;
    const int64_t *fund_off;
    float *grad_in;
    float *grad_w;
    int64_t n_common;              // N when grad_w is requested
    int32_t block_bins;            // bins per CTA
    int32_t max_cand;              // shared-memory candidate slots per CTA
    int32_t group;                 // spectra per CTA (grid.y = ceil(B / group))
    float *dw_partial;             // [groups][n_common] workspace when grid.y > 1 and grad_w is set
    int64_t blocks_per_spectrum;   // grid.x in per-spectrum mode
    uint8_t *active;               // [B][nblk] or nullptr: 1 where a bin block receives a contribution
    int64_t nblk;                  // bin blocks per spectrum in `active`
    int *nz_count;                 // [B]: fundamentals with a nonzero upstream gradient per spectrum
    int *nz_list;                  // [B][kBwdListCap]: those fundamentals (unordered) while they fit
    int *err;
};

// ---- kernel entry points (defined in the kernel translation units) ----
// 1D forward: kernel 0 = direct gather, 1 = greedy look-ahead gather, 2 = shared-memory
// windows staged by bulk copies (launched with a WinPlan as second parameter).
const void *fwd1d_kernel_f32(int forms, int whitening, int kernel);
const void *fwd1d_kernel_f16(int forms, int whitening, int kernel);
const void *fwd1d_kernel_bf16(int forms, int whitening, int kernel);
const void *fwd2d_kernel(int dtype);
const void *wait_selftest_kernel();
const void *fwd1d_opt_kernel(int dtype, int whitening, int H, int tail);
// 1D truncated tail (HS_FLAG_TRUNCATE_TAIL): fundamentals N_f <= n < N - 1, 256 threads per CTA,
// one CTA per generic tile and per one-order tile
const void *fwd1d_tail_kernel_f32(int forms, int whitening);
const void *fwd1d_tail_kernel_f16(int forms, int whitening);
const void *fwd1d_tail_kernel_bf16(int forms, int whitening);
constexpr int kTailThreads = 256;
constexpr int kTailTile = 1024;     // truncated-tail fundamentals per tile (kTailThreads x 4 per thread)
constexpr int kTail1Tile = 8192;    // one-order tail fundamentals per tile (eight rounds of kTailThreads x 4)
const void *bwd1d_kernel(int form, int dtype, int whitening);
const void *bwd_dw_reduce_kernel();
const void *bwd_mark_kernel(int form);

}  // namespace hs
