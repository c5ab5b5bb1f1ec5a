// Plan, validation, dispatch, CUDA-graph replay and autotuning behind the C ABI of hs.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include <cudaTypedefs.h>

#include "hs_fwd2d_sweep.cuh"
#include "hs_internal.cuh"
#include "hs_prewhiten.cuh"

using namespace hs;

namespace {

thread_local std::string g_last_cuda;

bool cuda_ok(cudaError_t e)
{
    if (e == cudaSuccess) return true;
    g_last_cuda = cudaGetErrorString(e);
    return false;
}

#define HS_CUDA(call)                                \
    do {                                             \
        if (!cuda_ok(call)) return HS_ERR_CUDA;      \
    } while (0)

constexpr uint32_t kKnownFlags = HS_FLAG_NO_MITIGATION | HS_FLAG_PER_SPECTRUM_NORM | HS_FLAG_WHITENING |
                                 HS_FLAG_AUTOTUNE | HS_FLAG_GRAPH | HS_FLAG_NO_DEVICE | HS_FLAG_CHECKED |
                                 HS_FLAG_TRUNCATE_TAIL;
constexpr size_t kWorkspaceBytes = 256;     // tile counter of the dynamic schedule
constexpr int kMaxChunks = 16;               // chunks of the pipelined host input
constexpr int kBwdBlockBins = 1024;   // must stay <= 32767 (int16 offsets)
constexpr int kBwdMaxGroups = 16;     // spectrum groups of the adjoint's dL/dw partial sums
constexpr int kBwdThreads = 256;
static_assert(kBwdBlockBins == 4 * kBwdThreads, "the adjoint's epilogue gives each thread four bins");

int elem_bytes(int dtype) { return dtype == HS_F32 ? 4 : 2; }

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Restores the calling thread's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && !cuda_ok(cudaSetDevice(dev))) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct GraphKey {
    const void *spectra, *w, *ws;
    hs_form_io s, g;
    bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

}  // namespace

struct hs_plan_s {
    hs_desc d{};
    int device = 0;
    bool no_device = false;
    int sms = 0;
    int path_bytes = 0;
    std::vector<int64_t> len, in_off, nf, fund_off, tile_start;
    std::vector<int64_t> nf_main, tail_tile_start;   // full-harmonic fundamentals; truncated-tail tiles
    std::vector<int64_t> tail1_tile_start;           // tiles of the tail's one-order fundamentals
    bool equal_lengths = false;   // 1D: every spectrum has one length (so one tile count)
    int64_t total_fund = 0, extent = 0, max_len = 0;
    int64_t f_lo = 0, f_hi = -1, z_lo = 0, z_hi = -1;
    hs_tuning tun{1, 256, 1, 0, 0, 0, 0, 0, 0};
    int l2_bytes = 0;
    WinPlan wplan{};
    // device tables
    int64_t *d_in_off = nullptr, *d_fund_off = nullptr, *d_tile_start = nullptr, *d_in_len = nullptr;
    int64_t *d_nf_main = nullptr, *d_tail_tile_start = nullptr, *d_tail1_tile_start = nullptr;
    int *d_err = nullptr;
    // graph replay
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey{};
    bool gvalid = false;
    std::mutex mu;
    // pipelined host input (hs_run_host): chunks of tiles with the input range their bins lie in
    // and the output range they write; each chunk launches on a tile prefix shifted to its
    // first tile (d_chunk_tile_start, kMaxChunks x (B+1))
    struct Chunk {
        int64_t t_a, t_b;        // tiles [t_a, t_b) of the main pass
        int64_t in_lo, in_hi;    // input elements [in_lo, in_hi) copied before the chunk runs
        int64_t out_lo, out_hi;  // outputs [out_lo, out_hi) the chunk completes
    };
    std::vector<Chunk> chunks;
    bool chunk_out = false;      // outputs can be copied back chunk by chunk (no truncated tail)
    int host_chunks = 0;         // requested chunk count (0: about 16 MiB of input per chunk)
    int64_t *d_chunk_tile_start = nullptr;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_start = nullptr, ev_done = nullptr, ev_in[kMaxChunks] = {}, ev_out[kMaxChunks] = {};
};

namespace {

// Fundamentals per tile: kernel 6 gives each fundamental one lane per form.
int64_t tile_fund(const hs_desc &d, const hs_tuning &t)
{
    if (t.kernel == 6 || t.kernel == 7) {
        const int64_t pass = (d.forms & 3) == (HS_FORM_SIMPLE | HS_FORM_GREEDY) ? t.threads / 2 : t.threads;
        return t.kernel == 7 ? 2 * pass : pass;
    }
    return static_cast<int64_t>(t.threads) * t.fund_per_thread;
}

// ---- 2D column sweep (kernel 2 of a 2D plan; schedule in hs_fwd2d_sweep.cuh) ----
constexpr int kSweepStaticSmem = 3072;          // static shared memory of the sweep kernel (upper bound)
constexpr int kSweepSmemLimit = 232448;         // 227 KiB opt-in per CTA
constexpr int64_t kSweepPrefixBands = 64;       // chains f < 64 Wb run whole in the prefix tasks

// Band width (anchor columns) when the tuning leaves it open: the two buffers (plane tile + the
// band's chain state) of a ~200-row plane at H = 8 then take ~206 KB for FP32 (64 columns) and
// ~209 KB for 16-bit storage (96 columns), one 512-thread CTA per SM.
// Band width of the column sweep when tuning.stage_kb is 0.  On the 201 x 2^21 plane, H = 8, 1024
// threads: FP32 112 columns 547 us (64: 790 us with 512 threads, 128: 640 us), FP16 176 columns
// 519 us (112: 534 us).
int sweep_default_wb(int dtype) { return dtype == HS_F32 ? 112 : 176; }

struct SweepGeom {
    bool ok = false;
    int Wb = 0, r_lo = 0, nr = 0, box_bytes = 0, buf_bytes = 0, nbuf = 0;
    int64_t f_s = 0, band_lo = 0, nbands = 0, n_prefix = 0;
    size_t state_bytes = 0, sync_bytes = 0;
};

// Geometry of the sweep with band width Wb and `threads` per CTA; ok = false where the sweep
// does not apply (checked plans, a row stride that is not a multiple of 16 bytes, more staged
// rows than one tensor-copy box holds, tiles beyond shared memory, nothing beyond the prefix).
SweepGeom sweep_geom(const hs_plan p, int Wb, int threads, int nbuf = 2, int64_t prefix_bands = kSweepPrefixBands)
{
    SweepGeom g;
    const hs_desc &d = p->d;
    if (d.dims != 2 || (d.flags & HS_FLAG_CHECKED) || p->f_hi < p->f_lo || threads < 32 || threads % 32) return g;
    const int eb = elem_bytes(d.dtype);
    if (Wb < 16 || Wb % 16 || Wb + 2 * kSweepHalo > kSweepMaxBox) return g;
    if ((d.n_freq * eb) % 16 || d.n_freq > (int64_t(1) << 30)) return g;
    // rows a chain can read: z0 + h z +- h for z in [z_lo, z_hi], h = 1..H
    const int64_t H = d.H;
    int64_t rmin = d.z0_row + p->z_lo - 1, rmax = d.z0_row + p->z_hi + 1;
    for (int64_t h = 2; h <= H; ++h) {
        rmin = std::min(rmin, d.z0_row + h * p->z_lo - h);
        rmax = std::max(rmax, d.z0_row + h * p->z_hi + h);
    }
    rmin = std::max<int64_t>(rmin, 0);
    rmax = std::min<int64_t>(rmax, d.n_rows - 1);
    const int64_t nr = rmax - rmin + 1;
    if (nr < 3 || nr > kSweepMaxBox) return g;
    const int64_t nz = p->z_hi - p->z_lo + 1;
    const int64_t box = nr * (Wb + 2 * kSweepHalo) * eb;
    const int64_t buf = (box + 127) / 128 * 128;   // one buffer: the band's staged plane tile
    if (nbuf < 2 || nbuf > kSweepMaxStages || nbuf * buf + kSweepStaticSmem > kSweepSmemLimit) return g;
    const int64_t f_s = std::max<int64_t>(p->f_lo, prefix_bands * Wb);
    if (f_s > p->f_hi) return g;
    const int compute = threads - 64;   // warps 0 and 1 control and publish
    if (compute < 32) return g;
    g.Wb = Wb;
    g.r_lo = static_cast<int>(rmin);
    g.nr = static_cast<int>(nr);
    g.box_bytes = static_cast<int>(box);
    g.buf_bytes = static_cast<int>(buf);
    g.nbuf = nbuf;
    g.f_s = f_s;
    g.band_lo = f_s / Wb;
    g.nbands = H * p->f_hi / Wb - g.band_lo + 1;
    g.n_prefix = ((f_s - p->f_lo) * nz + compute - 1) / compute;
    if (nz * (p->f_hi - f_s + 1) >= (int64_t(1) << 31)) return g;   // the kernel indexes the state in 32 bits
    g.state_bytes = static_cast<size_t>(nz * (p->f_hi - f_s + 1)) * 16;
    g.sync_bytes = (static_cast<size_t>(2 + g.nbands) * 4 + 255) / 256 * 256;
    g.ok = true;
    return g;
}

// Band width for tuning.stage_kb = 0: the default, or the widest narrower multiple of 16 that the
// plane takes (on a narrow plane no chain may lie beyond 64 default band widths).
int sweep_auto_wb(const hs_plan p, int threads, int nbuf, int producers)
{
    for (int wb = sweep_default_wb(p->d.dtype); wb >= 16; wb -= 16)
        if (sweep_geom(p, wb, threads, nbuf, kSweepPrefixBands * std::max(1, producers)).ok) return wb;
    return sweep_default_wb(p->d.dtype);
}

// Forward workspace: the dynamic schedule's tile counter (1D); the sweep's chain state and band
// flags (2D), sized for the narrowest band (16 columns: the most bands; any band width the sweep
// can take, 16 can take too).
// 1D with whitening: the forward writes the whitened input fl32(w[j] p[j]) (FP32, at the input's
// offsets) into the workspace after the tile counter, then runs the plain pass on it.
constexpr size_t kWhitenedOffset = kWorkspaceBytes;
size_t whitened_bytes(const hs_plan p)
{
    if (p->d.dims != 1 || !(p->d.flags & HS_FLAG_WHITENING)) return 0;
    return (static_cast<size_t>(p->extent) * 4 + 255) / 256 * 256;
}

size_t fwd_workspace_bytes(const hs_plan p)
{
    if (p->d.dims == 1) return kWorkspaceBytes + whitened_bytes(p);
    const SweepGeom n = sweep_geom(p, 16, kSweepThreads);   // the most bands and the most sweep chains
    return n.ok ? n.state_bytes + n.sync_bytes : 0;
}

// Adjoint with dL/dw: spectra are split into groups summed by different CTAs; each group's
// partial dL/dw (N floats) lives in the workspace and a final pass adds them in order.
int bwd_groups(const hs_plan p)
{
    if (p->d.dims != 1 || !(p->d.flags & HS_FLAG_WHITENING)) return 1;
    return static_cast<int>(std::min<int64_t>(p->d.num_spectra, kBwdMaxGroups));
}

// Adjoint workspace: [dL/dw partials: groups x N floats, when there is more than one group]
// [active-block flags: B x ceil(max N / block) bytes], each part 256-byte aligned.
int64_t bwd_nblk(const hs_plan p) { return (p->max_len + kBwdBlockBins - 1) / kBwdBlockBins; }

size_t bwd_partial_bytes(const hs_plan p)
{
    const int g = bwd_groups(p);
    const size_t b = g > 1 ? static_cast<size_t>(g) * static_cast<size_t>(p->len[0]) * sizeof(float) : 0;
    return (b + 255) / 256 * 256;
}

size_t bwd_flag_bytes(const hs_plan p)
{
    const size_t flags = static_cast<size_t>(p->d.num_spectra) * static_cast<size_t>(bwd_nblk(p));
    return (flags + 255) / 256 * 256;
}

// ... then the per-spectrum nonzero counts (B ints) and lists (B x kBwdListCap ints)
size_t bwd_workspace_bytes(const hs_plan p)
{
    if (p->d.dims != 1) return 0;
    const size_t B = static_cast<size_t>(p->d.num_spectra);
    return bwd_partial_bytes(p) + bwd_flag_bytes(p) + (B * 4 + 255) / 256 * 256 + B * 4 * kBwdListCap;
}
void make_win_plan(hs_plan p);

// Chunks of the pipelined host input (1D).  Fundamental n reads bins up to H n + H, so the
// tiles ending at fundamental n_b need the input only up to H n_b + 1 (plus a margin for the
// 16-byte-rounded window copies); one spectrum is cut into tile ranges, a batch into groups of
// whole spectra.  By default about 16 MiB of input per chunk, at most 8 (hs_plan_set_host_chunks
// sets the count, up to kMaxChunks); a batch whose spectra do not lie in increasing order is one
// chunk.
void make_chunks(hs_plan p)
{
    p->chunks.clear();
    p->chunk_out = !(p->d.flags & HS_FLAG_TRUNCATE_TAIL);
    if (p->d.dims != 1) return;
    const int64_t B = static_cast<int64_t>(p->nf.size());
    const int64_t T = tile_fund(p->d, p->tun);
    const int64_t H = p->d.H;
    const int64_t eb = elem_bytes(p->d.dtype);
    bool ordered = true;
    for (int64_t s = 0; s + 1 < B; ++s)
        if (p->in_off[s] + p->len[s] > p->in_off[s + 1]) ordered = false;
    const int64_t want = p->host_chunks > 0 ? p->host_chunks
                                            : std::max<int64_t>(1, std::min<int64_t>(8, p->extent * eb / (16ll << 20)));
    const int64_t K = ordered ? want : 1;
    const int64_t total = p->tile_start[B];
    if (K == 1 || total == 0) {
        p->chunks.push_back({0, total, 0, p->extent, 0, p->total_fund});
        return;
    }
    if (B == 1) {
        const int64_t base = p->in_off[0], len = p->len[0], nf = p->nf_main[0];
        int64_t lo = base;
        // decreasing chunk sizes (K : K-1 : ... : 1): the last chunk, whose pass and output copies
        // follow the last input copy, is the smallest
        const int64_t wsum = K * (K + 1) / 2;
        auto edge = [&](int64_t c) { return total * (c * K - c * (c - 1) / 2) / wsum; };   // sum of the first c weights
        for (int64_t c = 0; c < K; ++c) {
            const int64_t t_a = edge(c), t_b = edge(c + 1);
            if (t_b <= t_a) continue;
            const int64_t n_b = std::min(nf, t_b * T);
            int64_t need = c + 1 == K ? len : std::min(len, H * n_b + 1 + 32);
            int64_t hi = base + need;
            if (c + 1 < K) hi = std::min(p->extent, (hi + 15) / 16 * 16);
            else hi = p->extent;
            p->chunks.push_back({t_a, t_b, lo, std::max(lo, hi), p->fund_off[0] + t_a * T, p->fund_off[0] + n_b});
            lo = std::max(lo, hi);
        }
        return;
    }
    // whole spectra per chunk, about extent / K elements each
    int64_t s0 = 0;
    for (int64_t c = 0; c < K && s0 < B; ++c) {
        int64_t s1 = s0 + 1;
        const int64_t goal = p->extent * (c + 1) / K;
        while (s1 < B && (c + 1 == K || p->in_off[s1] + p->len[s1] <= goal)) ++s1;
        if (c + 1 == K) s1 = B;
        const int64_t lo = s0 == 0 ? 0 : p->in_off[s0];
        const int64_t hi = s1 == B ? p->extent : p->in_off[s1];
        p->chunks.push_back({p->tile_start[s0], p->tile_start[s1], lo, hi, p->fund_off[s0], p->fund_off[s1]});
        s0 = s1;
    }
}

void compute_tiles(hs_plan p)
{
    const int64_t T = tile_fund(p->d, p->tun);
    const size_t B = p->nf.size();
    p->tile_start.assign(B + 1, 0);
    // the main kernels cover the fundamentals with all H orders; the truncated tail has its own tiles
    for (size_t s = 0; s < B; ++s) p->tile_start[s + 1] = p->tile_start[s] + (p->nf_main[s] + T - 1) / T;
    // the truncated tail in two parts: N_f <= n < min(N - 1, n1), where the orders that fit vary, and
    // max(n1, N_f) <= n < N - 1, where both forms keep order 1 only (n1 = floor((N - 1) / 2) + 1)
    p->tail_tile_start.assign(B + 1, 0);
    p->tail1_tile_start.assign(B + 1, 0);
    for (size_t s = 0; s < B; ++s) {
        const int64_t n1 = (p->len[s] - 1) / 2 + 1;
        const int64_t g = std::max<int64_t>(0, std::min(p->nf[s], n1) - p->nf_main[s]);
        const int64_t o = std::max<int64_t>(0, p->nf[s] - std::max(n1, p->nf_main[s]));
        p->tail_tile_start[s + 1] = p->tail_tile_start[s] + (g + kTailTile - 1) / kTailTile;
        p->tail1_tile_start[s + 1] = p->tail1_tile_start[s] + (o + kTail1Tile - 1) / kTail1Tile;
    }
    make_win_plan(p);
    make_chunks(p);
}

hs_status upload_tiles(hs_plan p)
{
    if (p->no_device || p->d.dims != 1) return HS_OK;
    HS_CUDA(cudaMemcpy(p->d_tile_start, p->tile_start.data(), sizeof(int64_t) * p->tile_start.size(),
                       cudaMemcpyHostToDevice));
    if (p->d_chunk_tile_start) {
        const size_t B1 = p->tile_start.size();
        std::vector<int64_t> shifted(p->chunks.size() * B1);
        for (size_t c = 0; c < p->chunks.size(); ++c)
            for (size_t s = 0; s < B1; ++s) shifted[c * B1 + s] = p->tile_start[s] - p->chunks[c].t_a;
        HS_CUDA(cudaMemcpy(p->d_chunk_tile_start, shifted.data(), sizeof(int64_t) * shifted.size(),
                           cudaMemcpyHostToDevice));
    }
    return HS_OK;
}

constexpr int kMaxDynSmem = 232448 - kWinStaticSmem;   // 227 KiB opt-in per CTA, minus static

hs_status validate_tuning(const hs_plan p, const hs_tuning *t)
{
    if (!t) return HS_ERR_INVALID_ARG;
    if (t->kernel < 0 || t->kernel > 7) return HS_ERR_INVALID_ARG;
    if (t->threads < 64 || (t->threads % 32) != 0) return HS_ERR_INVALID_ARG;
    if (t->threads > (t->kernel == 2 ? 512 : 256)) return HS_ERR_INVALID_ARG;
    if (t->kernel == 2 && (p->d.flags & HS_FLAG_WHITENING)) return HS_ERR_UNSUPPORTED;
    if (t->fund_per_thread != (t->kernel == 3 ? 2 : 1)) return HS_ERR_INVALID_ARG;
    if (t->kernel == 3 && t->dynamic) return HS_ERR_INVALID_ARG;
    if (t->ctas_per_sm < 0 || t->ctas_per_sm > 32) return HS_ERR_INVALID_ARG;
    if (t->dynamic != 0 && t->dynamic != 1) return HS_ERR_INVALID_ARG;
    // prefetch bit 0: the whole input into L2 at launch when it fits in part of L2 (kernels 2, 6, 7);
    // bit 1: the tiles of each spectrum prefetch the next spectrum (every kernel but 2)
    if (t->prefetch < 0 || t->prefetch > 3) return HS_ERR_INVALID_ARG;
    if ((t->prefetch & 1) && t->kernel != 2 && t->kernel != 6 && t->kernel != 7) return HS_ERR_INVALID_ARG;
    if ((t->prefetch & 2) && t->kernel == 2) return HS_ERR_INVALID_ARG;
    if (t->kernel != 2 && t->producers != 0) return HS_ERR_INVALID_ARG;
    if (t->kernel == 2) {
        if (p->d.flags & HS_FLAG_WHITENING) return HS_ERR_UNSUPPORTED;
        if (t->dynamic) return HS_ERR_INVALID_ARG;
        if (t->stages < 2 || t->stages > 16 || t->stage_kb < 1) return HS_ERR_INVALID_ARG;
        if (t->producers < 1 || t->producers > 8 || t->producers > t->stages) return HS_ERR_INVALID_ARG;
        if (t->threads + 32 * t->producers > 640) return HS_ERR_INVALID_ARG;
        const int64_t bb = static_cast<int64_t>(t->stage_kb) * 1024;
        if (bb < win_bytes(p->d.H, t->threads, elem_bytes(p->d.dtype))) return HS_ERR_INVALID_ARG;
        if (bb * t->stages > kMaxDynSmem) return HS_ERR_INVALID_ARG;
    } else if (t->dynamic && t->ctas_per_sm == 0) {
        return HS_ERR_INVALID_ARG;
    }
    return HS_OK;
}

// Ring plan of the window kernel.
void make_win_plan(hs_plan p)
{
    WinPlan &w = p->wplan;
    w = WinPlan{};
    const hs_tuning &t = p->tun;
    if (t.kernel != 2) return;
    w.T = t.threads;
    w.nslot = t.stages;
    w.nprod = t.producers;
    w.slot_bytes = t.stage_kb * 1024;
    w.extent = p->extent;
    w.pf_chunk = 0;   // set at launch (depends on the grid)
}

hs_tuning default_tuning(const hs_plan p)
{
    // Fused plans whose input exceeds L2 (batches of spectra streaming from DRAM): two
    // fundamentals per thread (kernel 3, 128-thread CTAs) keep the most gathers in flight --
    // 18.3 ms vs 24.2 ms (kernel 0) on 2048 spectra of 2^20..2^23 bins, H = 16, FP32; with 16-bit
    // storage each spectrum's tiles also prefetch the next spectrum into L2 (15.2 vs 15.8 ms).
    if (p->l2_bytes > 0 && p->extent * elem_bytes(p->d.dtype) > p->l2_bytes &&
        (p->d.forms & 3) == 3 && !(p->d.flags & HS_FLAG_WHITENING))
        return hs_tuning{3, 128, 2, 0, 0, 0, 0, (p->d.dtype != HS_F32 && p->d.num_spectra > 1) ? 2 : 0, 0};
    // Measured on the 2^23-bin H = 32 spectrum (GB300): FP32 without whitening runs fastest on
    // the paired-lane kernel 6 in 128-thread CTAs (fused 42.9 us vs 43.6 us with 256 threads and
    // 45.3 us on kernel 0; an L2 prefetch of the whole input first costs 2.5 us); with whitening or
    // 16-bit storage the direct kernel 0 is as fast or faster (kernel 6 on FP16: 33.3 vs 32.8 us).
    // HS_FLAG_AUTOTUNE times the alternatives per plan.
    if (p->d.dtype == HS_F32 && !(p->d.flags & HS_FLAG_WHITENING)) return hs_tuning{6, 128, 1, 0, 0, 0, 0, 0, 0};
    return hs_tuning{0, p->d.dtype == HS_F32 ? 256 : 128, 1, 0, 0, 0, 0, 0, 0};
}

hs_status ensure_bwd_smem(const void *fn, size_t bytes)
{
    if (bytes <= 48 * 1024) return HS_OK;
    HS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)));
    return HS_OK;
}

// Kernels whose dynamic shared-memory limit has been raised, per device (the attribute belongs to
// the device the call is made on).
std::mutex g_attr_mu;
std::vector<std::pair<int, const void *>> g_attr_set;

bool attr_is_set(const void *fn, int *device)
{
    if (cudaGetDevice(device) != cudaSuccess) *device = -1;
    return std::find(g_attr_set.begin(), g_attr_set.end(), std::make_pair(*device, fn)) != g_attr_set.end();
}

hs_status ensure_dyn_smem(const void *fn)
{
    std::lock_guard<std::mutex> lk(g_attr_mu);
    int dev = 0;
    if (attr_is_set(fn, &dev)) return HS_OK;
    HS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
    g_attr_set.emplace_back(dev, fn);
    return HS_OK;
}

const void *fwd1d_kernel(int dtype, int forms, int whitening, int kernel)
{
    switch (dtype) {
    case HS_F32: return fwd1d_kernel_f32(forms, whitening, kernel);
    case HS_F16: return fwd1d_kernel_f16(forms, whitening, kernel);
    case HS_BF16: return fwd1d_kernel_bf16(forms, whitening, kernel);
    }
    return nullptr;
}

void free_plan(hs_plan p)
{
    if (!p) return;
    if (!p->no_device) {
        DeviceGuard g(p->device);
        if (p->gexec) cudaGraphExecDestroy(p->gexec);
        if (p->cap) cudaStreamDestroy(p->cap);
        cudaFree(p->d_in_off);
        cudaFree(p->d_fund_off);
        cudaFree(p->d_tile_start);
        cudaFree(p->d_nf_main);
        cudaFree(p->d_tail_tile_start);
        cudaFree(p->d_tail1_tile_start);
        cudaFree(p->d_in_len);
        cudaFree(p->d_err);
        cudaFree(p->d_chunk_tile_start);
        if (p->h2d) cudaStreamDestroy(p->h2d);
        if (p->d2h) cudaStreamDestroy(p->d2h);
        if (p->ev_start) cudaEventDestroy(p->ev_start);
        if (p->ev_done) cudaEventDestroy(p->ev_done);
        for (int i = 0; i < kMaxChunks; ++i) {
            if (p->ev_in[i]) cudaEventDestroy(p->ev_in[i]);
            if (p->ev_out[i]) cudaEventDestroy(p->ev_out[i]);
        }
    }
    delete p;
}

hs_status check_io(const hs_plan p, const hs_form_io *io, bool greedy)
{
    if (!io || !io->mu || !io->sigma || !io->snr || !io->best_h) return HS_ERR_INVALID_ARG;
    if (!aligned(io->mu, 4) || !aligned(io->sigma, 4) || !aligned(io->snr, 4)) return HS_ERR_INVALID_ARG;
    if (io->argmax && !aligned(io->argmax, 8)) return HS_ERR_INVALID_ARG;
    if (io->path) {
        if (!greedy) return HS_ERR_INVALID_ARG;
        if (!aligned(io->path, p->path_bytes)) return HS_ERR_INVALID_ARG;
    }
    return HS_OK;
}

FormArgs to_form_args(const hs_form_io *io)
{
    FormArgs f{};
    if (!io) return f;
    f.mu = io->mu;
    f.sigma = io->sigma;
    f.snr = io->snr;
    f.best_h = io->best_h;
    f.path = io->path;
    f.argmax = reinterpret_cast<unsigned long long *>(io->argmax);
    return f;
}

const void *fwd1d_tail_kernel(int dtype, int forms, int whitening)
{
    switch (dtype) {
    case HS_F32: return fwd1d_tail_kernel_f32(forms, whitening);
    case HS_F16: return fwd1d_tail_kernel_f16(forms, whitening);
    case HS_BF16: return fwd1d_tail_kernel_bf16(forms, whitening);
    }
    return nullptr;
}

// Launch of a 1D forward kernel; with `after_reset` it may start while k_fwd_reset (enqueued just
// before it) still runs -- every 1D forward kernel waits (griddepcontrol.wait) before it touches
// what the reset writes.
hs_status launch_fwd(const void *fn, dim3 grid, dim3 block, void **args, size_t smem, cudaStream_t st,
                     bool after_reset)
{
    if (!after_reset) {
        HS_CUDA(cudaLaunchKernel(fn, grid, block, args, smem, st));
        return HS_OK;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HS_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
    return HS_OK;
}

// The truncated tail (HS_FLAG_TRUNCATE_TAIL): fundamentals N_f <= n < N - 1, after the main kernel,
// in one launch: the generic tiles (below n1 = floor((N - 1) / 2) + 1) and the one-order tiles.
hs_status launch_tail(const hs_plan p, const Fwd1DArgs &main_args, cudaStream_t st, bool prewhitened = false)
{
    if (!(p->d.flags & HS_FLAG_TRUNCATE_TAIL)) return HS_OK;
    const int64_t ctas = main_args.tail_tiles + main_args.tail1_tiles;
    if (ctas <= 0) return HS_OK;
    if (ctas > 0x7fffffff) return HS_ERR_UNSUPPORTED;
    // on the pre-whitened copy the tail reads plain FP32
    const void *fn = prewhitened ? fwd1d_tail_kernel(HS_F32, p->d.forms & 3, 0)
                                 : fwd1d_tail_kernel(p->d.dtype, p->d.forms & 3, (p->d.flags & HS_FLAG_WHITENING) ? 1 : 0);
    if (!fn) return HS_ERR_UNSUPPORTED;
    Fwd1DArgs a = main_args;
    a.tile_counter = nullptr;
    a.pf_chunk = 0;
    void *args[] = {&a};
    HS_CUDA(cudaLaunchKernel(fn, dim3(static_cast<unsigned>(ctas)), dim3(kTailThreads), args, 0, st));
    return HS_OK;
}

// The sweep kernel's dynamic shared-memory limit: the per-CTA opt-in maximum less its static
// shared memory (set once per kernel).
hs_status ensure_sweep_smem(const void *fn)
{
    std::lock_guard<std::mutex> lk(g_attr_mu);
    int dev = 0;
    if (attr_is_set(fn, &dev)) return HS_OK;
    cudaFuncAttributes fa{};
    HS_CUDA(cudaFuncGetAttributes(&fa, fn));
    if (fa.sharedSizeBytes > static_cast<size_t>(kSweepStaticSmem)) return HS_ERR_UNSUPPORTED;
    HS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSweepSmemLimit - static_cast<int>(fa.sharedSizeBytes)));
    g_attr_set.emplace_back(dev, fn);
    return HS_OK;
}

// cuTensorMapEncodeTiled from the driver, through the runtime (no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

// The 2D sweep: reset the ticket / band flags, describe the plane to the tensor copies, launch a
// persistent grid.
hs_status launch_sweep(const hs_plan p, const Fwd2DArgs &a, const SweepGeom &g, void *ws, cudaStream_t st)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return HS_ERR_UNSUPPORTED;
    const int eb = elem_bytes(p->d.dtype);
    const CUtensorMapDataType dt = p->d.dtype == HS_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : p->d.dtype == HS_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(p->d.n_freq), static_cast<cuuint64_t>(p->d.n_rows)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(p->d.n_freq) * eb};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(g.Wb + 2 * kSweepHalo), static_cast<cuuint32_t>(g.nr)};
    const cuuint32_t estr[2] = {1, 1};
    CUtensorMap map;
    if (enc(&map, dt, 2, const_cast<void *>(a.plane), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return HS_ERR_CUDA;
    Sweep2DArgs s{};
    s.a = a;
    s.f_s = g.f_s;
    s.n_prefix = g.n_prefix;
    s.band_lo = g.band_lo;
    s.nbands = g.nbands;
    s.Wb = g.Wb;
    s.r_lo = g.r_lo;
    s.nr = g.nr;
    s.box_bytes = g.box_bytes;
    s.nfs = p->f_hi - g.f_s + 1;
    s.buf_bytes = g.buf_bytes;
    s.nbuf = g.nbuf;
    s.state = static_cast<int4 *>(ws);
    s.sync = reinterpret_cast<unsigned *>(static_cast<uint8_t *>(ws) + g.state_bytes);
    HS_CUDA(cudaMemsetAsync(s.sync, 0, sizeof(unsigned) * static_cast<size_t>(2 + g.nbands), st));
    const void *fn = fwd2d_sweep_kernel(p->d.dtype);
    if (!fn) return HS_ERR_UNSUPPORTED;
    hs_status es = ensure_sweep_smem(fn);
    if (es != HS_OK) return es;
    const size_t smem = static_cast<size_t>(g.nbuf) * g.buf_bytes;
    const int threads = p->tun.threads;
    int per_sm = p->tun.ctas_per_sm;
    if (per_sm <= 0) {
        HS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
        per_sm = std::max(per_sm, 1);
    }
    const int64_t grid = std::min<int64_t>(static_cast<int64_t>(per_sm) * p->sms, g.n_prefix + g.nbands);
    void *args[] = {&map, &s};
    HS_CUDA(cudaLaunchKernel(fn, dim3(static_cast<unsigned>(grid)), dim3(threads), args, smem, st));
    return HS_OK;
}

// Band width of the sweep under the plan's tuning (stage_kb = width / 16; 0 = default) and its
// buffers (stages; 0 = 2).
int sweep_stages(const hs_plan p) { return p->tun.stages > 0 ? p->tun.stages : 2; }
int sweep_wb(const hs_plan p)
{
    return p->tun.stage_kb > 0 ? 16 * p->tun.stage_kb
                               : sweep_auto_wb(p, p->tun.threads, sweep_stages(p), p->tun.producers);
}
// Chains f < prefix bands x Wb run whole in registers (prefix tasks); tuning.producers scales the
// default 64 bands (0 or 1: 64, k: 64 k).
int64_t sweep_prefix(const hs_plan p) { return kSweepPrefixBands * std::max(1, p->tun.producers); }

// Enqueue the forward pass (memsets + the main kernel + the truncated tail's) on `st`.
// chunk >= 0 (1D): only the tiles of that chunk of the pipelined host input, on the tile prefix
// shifted to its first tile, without the argmax reset (done once before the first chunk), the L2
// prefetches (their input may not have arrived yet) or, but for the last chunk, the tail.
hs_status enqueue_fwd(hs_plan p, const void *spectra, const float *w, const hs_form_io *simple,
                      const hs_form_io *greedy, void *ws, cudaStream_t st, int chunk = -1, bool prewhiten = false)
{
    const int64_t B = p->d.dims == 1 ? p->d.num_spectra : 1;
    if (p->d.dims == 2) {
        if (greedy && greedy->argmax) HS_CUDA(cudaMemsetAsync(greedy->argmax, 0, sizeof(uint64_t), st));
        Fwd2DArgs a{};
        a.plane = spectra;
        a.n_freq = p->d.n_freq;
        a.n_rows = p->d.n_rows;
        a.z0_row = p->d.z0_row;
        a.H = p->d.H;
        a.f_lo = p->f_lo;
        a.nff = p->f_hi - p->f_lo + 1;
        a.z_lo = p->z_lo;
        a.nz = p->z_hi - p->z_lo + 1;
        a.checked = (p->d.flags & HS_FLAG_CHECKED) ? 1 : 0;
        a.g = to_form_args(greedy);
        a.err = p->d_err;
        if (p->tun.kernel == 2 && ws) {
            const SweepGeom g = sweep_geom(p, sweep_wb(p), p->tun.threads, sweep_stages(p), sweep_prefix(p));
            if (g.ok) return launch_sweep(p, a, g, ws, st);
        }
        // kernel 2 without a workspace runs as kernel 1 (the outputs are the same bit for bit)
        const int threads = 256;
        const int64_t ftiles = (a.nff + threads - 1) / threads;
        // tuning.kernel 1 (2D): z rows fastest, while the f-tiles fit in grid.y
        a.zfast = (p->tun.kernel != 0 && ftiles <= 65535) ? 1 : 0;
        dim3 grid = a.zfast ? dim3(static_cast<unsigned>(a.nz), static_cast<unsigned>(ftiles))
                            : dim3(static_cast<unsigned>(ftiles), static_cast<unsigned>(a.nz));
        void *args[] = {&a};
        HS_CUDA(cudaLaunchKernel(fwd2d_kernel(p->d.dtype), grid, dim3(threads), args, 0, st));
        return HS_OK;
    }
    const hs_tuning &t = p->tun;
    Fwd1DArgs a{};
    a.x = spectra;
    a.w = w;
    a.in_off = p->d_in_off;
    a.fund_off = p->d_fund_off;
    a.nf_main = p->d_nf_main;
    a.tail_tile_start = p->d_tail_tile_start;
    a.tail_tiles = p->tail_tile_start.empty() ? 0 : p->tail_tile_start.back();
    a.tail1_tile_start = p->d_tail1_tile_start;
    a.tail1_tiles = p->tail1_tile_start.empty() ? 0 : p->tail1_tile_start.back();
    a.tile_start = p->d_tile_start;
    a.in_len = p->d_in_len;
    a.B = static_cast<int32_t>(p->d.num_spectra);
    // one tile count for every spectrum: the kernels find a tile's spectrum by a division (below
    // 2^22 tiles a single-precision estimate is within one of the quotient)
    if (p->equal_lengths && p->tile_start.back() < (int64_t(1) << 22) && p->tail_tile_start.back() < (int64_t(1) << 22) &&
        p->tail1_tile_start.back() < (int64_t(1) << 22)) {
        a.tiles_per_spec = static_cast<uint32_t>(p->tile_start.back() / p->d.num_spectra);
        a.tail_tiles_per_spec = static_cast<uint32_t>(p->tail_tile_start.back() / p->d.num_spectra);
        a.tail1_tiles_per_spec = static_cast<uint32_t>(p->tail1_tile_start.back() / p->d.num_spectra);
        a.inv_tiles_per_spec = a.tiles_per_spec ? 1.0f / static_cast<float>(a.tiles_per_spec) : 0.f;
    }
    a.H = p->d.H;
    a.mitigation = (p->d.flags & HS_FLAG_NO_MITIGATION) ? 0 : 1;
    a.per_spectrum_norm = (p->d.flags & HS_FLAG_PER_SPECTRUM_NORM) ? 1 : 0;
    a.path_bytes = p->path_bytes;
    a.checked = (p->d.flags & HS_FLAG_CHECKED) ? 1 : 0;
    a.fund_per_thread = t.fund_per_thread;
    a.total_tiles = p->tile_start.back();
    a.extent = p->extent;
    a.elem_bytes = elem_bytes(p->d.dtype);
    a.pf_next = (t.prefetch & 2) ? 1 : 0;
    a.s = to_form_args(simple);
    a.g = to_form_args(greedy);
    a.err = p->d_err;
    const bool last = chunk < 0 || chunk + 1 == static_cast<int>(p->chunks.size());
    if (chunk >= 0) {
        const auto &c = p->chunks[chunk];
        a.tile_start = p->d_chunk_tile_start + static_cast<int64_t>(chunk) * (B + 1);
        a.total_tiles = c.t_b - c.t_a;
        a.pf_next = 0;
    }
    if ((p->d.forms & 3) == 0) return HS_OK;   // the optimal form runs through hs_run_optimal
    // a whole pass of a whitening plan given a workspace (prewhiten) first writes the whitened
    // input into it and then runs the plain FP32 pass on that copy: two gathers per loaded value
    // (w[j] and p[j]) become one.  The copy's float4 stores need a 16-byte aligned workspace; with
    // another, the pass multiplies as it loads.
    const bool whiten = (p->d.flags & HS_FLAG_WHITENING) != 0;
    const bool pre = prewhiten && whiten && ws && aligned(ws, 16) && chunk < 0 && t.kernel != 2;
    if (pre) {
        a.x = static_cast<const unsigned char *>(ws) + kWhitenedOffset;
        a.w = nullptr;
        a.elem_bytes = 4;
    }
    const void *fn = fwd1d_kernel(pre ? HS_F32 : p->d.dtype, p->d.forms & 3, (whiten && !pre) ? 1 : 0, t.kernel);
    if (!fn) return HS_ERR_UNSUPPORTED;
    // a whole pass clears the argmax keys (and the dynamic schedule's counter) with k_fwd_reset,
    // which the pass may overlap; a chunk of hs_run_host relies on the clear before its first chunk
    unsigned long long *s_key = simple ? reinterpret_cast<unsigned long long *>(simple->argmax) : nullptr;
    unsigned long long *g_key = greedy ? reinterpret_cast<unsigned long long *>(greedy->argmax) : nullptr;
    const bool dyn = t.kernel != 2 && t.dynamic && ws;
    bool after_reset = false;
    if (pre) {
        // the copy also clears the keys and the counter; the pass waits for the whole copy
        const int64_t N = p->len[0];
        const int64_t chunks = (N + 1023) / 1024 * B;
        const unsigned grid_w = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(chunks, 8ll * p->sms)));
        float *X = reinterpret_cast<float *>(static_cast<unsigned char *>(ws) + kWhitenedOffset);
        unsigned long long *cnt = dyn ? static_cast<unsigned long long *>(ws) : nullptr;
        const int32_t Bi = static_cast<int32_t>(B);
        if (p->d.dtype == HS_F32)
            k_prewhiten<float><<<grid_w, 256, 0, st>>>(static_cast<const float *>(spectra), w, X, p->d_in_off, Bi, N,
                                                        s_key, g_key, cnt);
        else if (p->d.dtype == HS_F16)
            k_prewhiten<__half><<<grid_w, 256, 0, st>>>(static_cast<const __half *>(spectra), w, X, p->d_in_off, Bi,
                                                         N, s_key, g_key, cnt);
        else
            k_prewhiten<__nv_bfloat16><<<grid_w, 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(spectra), w, X,
                                                                p->d_in_off, Bi, N, s_key, g_key, cnt);
        HS_CUDA(cudaGetLastError());
    } else if (chunk < 0 && (s_key || g_key || dyn)) {
        const int64_t rb = std::min<int64_t>(std::max<int64_t>((B + 255) / 256, 1), 64);
        k_fwd_reset<<<static_cast<unsigned>(rb), 256, 0, st>>>(s_key, g_key, (s_key || g_key) ? B : 0,
                                                              dyn ? static_cast<unsigned long long *>(ws) : nullptr);
        HS_CUDA(cudaGetLastError());
        after_reset = true;
    }
    if (t.kernel == 2) {
        const size_t smem = static_cast<size_t>(p->wplan.nslot) * p->wplan.slot_bytes;
        hs_status es = ensure_dyn_smem(fn);
        if (es != HS_OK) return es;
        const int block = t.threads + 32 * t.producers;
        int per_sm = t.ctas_per_sm;
        if (per_sm == 0) {
            HS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem));
            if (per_sm < 1) return HS_ERR_UNSUPPORTED;
        }
        int64_t grid = std::min<int64_t>(a.total_tiles, static_cast<int64_t>(per_sm) * p->sms);
        if (grid < 1) return last ? launch_tail(p, a, st) : HS_OK;
        WinPlan wp = p->wplan;
        const int64_t in_bytes = p->extent * elem_bytes(p->d.dtype);
        if (chunk < 0 && (t.prefetch & 1) && p->l2_bytes > 0 && in_bytes <= p->l2_bytes / 4)
            wp.pf_chunk = ((in_bytes + grid - 1) / grid + 15) / 16 * 16;
        void *args[] = {&a, &wp};
        hs_status ls = launch_fwd(fn, dim3(static_cast<unsigned>(grid)), dim3(block), args, smem, st, after_reset);
        if (ls != HS_OK) return ls;
        return last ? launch_tail(p, a, st) : HS_OK;
    }
    int64_t grid = a.total_tiles;
    if (t.ctas_per_sm > 0) grid = std::min<int64_t>(grid, static_cast<int64_t>(t.ctas_per_sm) * p->sms);
    if (chunk < 0 && (t.kernel == 6 || t.kernel == 7) && (t.prefetch & 1) && p->l2_bytes > 0 && grid > 0) {
        // an input that fits in half of L2 is prefetched there by the first CTAs, one share each
        const int64_t in_bytes = p->extent * a.elem_bytes;
        if (in_bytes <= p->l2_bytes / 2) {
            const int64_t ctas = std::min<int64_t>(grid, static_cast<int64_t>(p->sms) * 8);
            a.pf_bytes = in_bytes;
            a.pf_chunk = ((in_bytes + ctas - 1) / ctas + 15) / 16 * 16;
        }
    }
    if (t.dynamic) {
        a.tile_counter = static_cast<unsigned long long *>(ws);
        // every CTA draws all of its tiles from this counter, starting at 0 (cleared by k_fwd_reset
        // for a whole pass)
        if (chunk >= 0) HS_CUDA(cudaMemsetAsync(ws, 0, sizeof(unsigned long long), st));
    }
    if (grid > 0x7fffffff) return HS_ERR_UNSUPPORTED;
    if (grid >= 1) {
        void *args[] = {&a};
        hs_status ls = launch_fwd(fn, dim3(static_cast<unsigned>(grid)), dim3(t.threads), args, 0, st, after_reset);
        if (ls != HS_OK) return ls;
    }
    return last ? launch_tail(p, a, st, pre) : HS_OK;
}

// ---------------------------------------------------------------------------------------
// autotuner: times candidate launch shapes on a synthetic input shaped like the plan
// ---------------------------------------------------------------------------------------
__global__ void k_fill_noise(float *x, int64_t n, uint64_t seed)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        // splitmix64 of the index -> uniform in (0, 1] -> Exp(1) by inversion
        uint64_t z = seed + static_cast<uint64_t>(i) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const float u = (static_cast<float>(z >> 40) + 1.0f) * (1.0f / 16777216.0f);
        x[i] = -logf(u);
    }
}

__global__ void k_f32_to(const float *src, void *dst, int64_t n, int dtype)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (dtype == HS_F16) static_cast<__half *>(dst)[i] = __float2half_rn(src[i]);
        else static_cast<__nv_bfloat16 *>(dst)[i] = __float2bfloat16_rn(src[i]);
    }
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int, int, int>, hs_tuning> g_tune_cache;

hs_status autotune(hs_plan p)
{
    const auto key = std::make_tuple(p->device, p->d.H, p->d.forms, p->d.dtype,
                                     static_cast<int>(p->d.flags & (HS_FLAG_WHITENING | HS_FLAG_NO_MITIGATION)),
                                     static_cast<int>(std::ceil(std::log2(static_cast<double>(p->max_len)))),
                                     p->d.num_spectra > 1 ? 1 : 0, p->sms);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p->tun = it->second;
            compute_tiles(p);
            return upload_tiles(p);
        }
    }
    // sub-plan: spectra sampled evenly from the sorted lengths, packed, until the input reaches
    // eight times L2 (or the whole plan): the mix of lengths and the L2 behaviour of a schedule
    // (a static persistent grid drifts apart and thrashes L2 on large batches) resemble the plan's
    std::vector<int64_t> all(p->len);
    std::sort(all.begin(), all.end(), std::greater<int64_t>());
    const int64_t total_elems = std::accumulate(all.begin(), all.end(), int64_t(0));
    const int64_t want_elems = std::min<int64_t>(total_elems, 8 * static_cast<int64_t>(p->l2_bytes) / elem_bytes(p->d.dtype));
    size_t nsub = 1;
    while (nsub < all.size() && nsub < 1024) {
        int64_t e = 0;
        for (size_t i = 0; i < nsub; ++i) e += all[i * all.size() / nsub];
        if (e >= want_elems) break;
        ++nsub;
    }
    std::vector<int64_t> lens;
    for (size_t i = 0; i < nsub; ++i) lens.push_back(all[i * all.size() / nsub]);
    hs_desc sd = p->d;
    sd.num_spectra = static_cast<int64_t>(lens.size());
    sd.lengths = lens.data();
    sd.offsets = nullptr;
    sd.flags &= ~(HS_FLAG_AUTOTUNE | HS_FLAG_GRAPH | HS_FLAG_PER_SPECTRUM_NORM | HS_FLAG_CHECKED | HS_FLAG_TRUNCATE_TAIL);
    sd.forms &= 3;
    if (sd.flags & HS_FLAG_WHITENING) {
        for (auto &l : lens) l = lens[0];
    }
    hs_plan sp = nullptr;
    hs_status st = hs_plan_create(&sp, &sd, p->device);
    if (st != HS_OK) return st;
    const int64_t ext = sp->extent, F = sp->total_fund, H = sp->d.H;
    void *x = nullptr, *w = nullptr, *ws = nullptr, *outs = nullptr, *norm = nullptr, *tmp = nullptr;
    void *flush = nullptr;   // written before every timed run: candidates are timed on a cold L2
    int pf_next = 0, pf_all = 0;
    const int64_t ext_all = p->extent;
    bool big = false;
    const size_t flush_bytes = std::max<size_t>(2 * static_cast<size_t>(p->l2_bytes), size_t(64) << 20);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hs_status result = HS_OK;
    std::vector<hs_tuning> cands;
    float best_ms = 1e30f;
    hs_tuning best = p->tun;
    hs_form_io fs{}, fg{};
    const size_t out_bytes = static_cast<size_t>(F) * (4 + 1 + 4 + 1) + 256;
    if (!cuda_ok(cudaMalloc(&x, ext * elem_bytes(sd.dtype) + 64)) || !cuda_ok(cudaMalloc(&tmp, ext * 4 + 64)) ||
        !cuda_ok(cudaMalloc(&w, lens[0] * 4 + 64)) || !cuda_ok(cudaMalloc(&ws, fwd_workspace_bytes(sp))) ||
        !cuda_ok(cudaMalloc(&outs, out_bytes)) || !cuda_ok(cudaMalloc(&norm, 4 * H * 4)) ||
        !cuda_ok(cudaMalloc(&flush, flush_bytes)) ||
        !cuda_ok(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) || !cuda_ok(cudaEventCreate(&e0)) ||
        !cuda_ok(cudaEventCreate(&e1))) {
        result = HS_ERR_OOM;
        goto done;
    }
    {
        k_fill_noise<<<1024, 256, 0, s>>>(static_cast<float *>(tmp), ext, 0x2202128170ull);
        if (sd.dtype == HS_F32) cudaMemcpyAsync(x, tmp, ext * 4, cudaMemcpyDeviceToDevice, s);
        else k_f32_to<<<1024, 256, 0, s>>>(static_cast<const float *>(tmp), x, ext, sd.dtype);
        k_fill_noise<<<256, 256, 0, s>>>(static_cast<float *>(w), lens[0], 0x77ull);
        std::vector<float> hn(4 * H);
        hs_norm_exponential(HS_FORM_SIMPLE, 1, static_cast<int>(H), 1, 1.0, hn.data(), hn.data() + H);
        hs_norm_exponential(HS_FORM_GREEDY, 1, static_cast<int>(H), 1, 1.0, hn.data() + 2 * H, hn.data() + 3 * H);
        cudaMemcpyAsync(norm, hn.data(), 4 * H * 4, cudaMemcpyHostToDevice, s);
        char *o = static_cast<char *>(outs);
        auto a16 = [](int64_t v) { return (v + 15) / 16 * 16; };
        const int64_t o_sb = a16(4 * F), o_gs = a16(o_sb + F), o_gb = a16(o_gs + 4 * F);
        const float *nrm = static_cast<const float *>(norm);
        fs.mu = nrm; fs.sigma = nrm + H;
        fs.snr = reinterpret_cast<float *>(o);
        fs.best_h = reinterpret_cast<uint8_t *>(o + o_sb);
        fg.mu = nrm + 2 * H; fg.sigma = nrm + 3 * H;
        fg.snr = reinterpret_cast<float *>(o + o_gs);
        fg.best_h = reinterpret_cast<uint8_t *>(o + o_gb);
        fg.path = nullptr;
        if (!cuda_ok(cudaStreamSynchronize(s))) { result = HS_ERR_CUDA; goto done; }
    }
    for (int threads : {64, 128, 256})
        for (int prod : {2, 4, 8}) {
            const int kb = static_cast<int>((win_bytes(sp->d.H, threads, elem_bytes(sp->d.dtype)) + 1023) / 1024);
            for (int total_kb : {100, 200}) {
                const int slots = std::min(16, total_kb / kb);
                hs_tuning t{2, threads, 1, 0, 0, slots, kb, 0, prod};
                if (validate_tuning(sp, &t) == HS_OK) cands.push_back(t);
            }
        }
    // the next-spectrum prefetch (prefetch bit 1) only matters with several spectra, and only pays
    // with 16-bit storage: on the 2048-spectrum FP32 batch it ran 19.9 ms against 18.5 ms without,
    // although the 1 GB sub-plan ranked it first.  The whole-input prefetch (bit 0, kernels 6 and
    // 7) only matters when the input fits in half of L2.
    pf_next = (sd.num_spectra > 1 && sd.dtype != HS_F32) ? 2 : 0;
    pf_all = ext * elem_bytes(sd.dtype) <= p->l2_bytes / 2 ? 1 : 0;
    for (int threads : {64, 128, 256})
        for (int pf : {0, pf_next}) {
            hs_tuning t{3, threads, 2, 0, 0, 0, 0, pf, 0};
            if (validate_tuning(sp, &t) == HS_OK) cands.push_back(t);
            if (!pf_next) break;
        }
    // a static persistent grid drifts apart over a long pass and thrashes L2: on 2048 spectra
    // (32 GB) it ran 30% slower than one CTA per tile although it won on a 1 GB sample, so it
    // is not a candidate for plans larger than L2
    big = ext_all * elem_bytes(p->d.dtype) > static_cast<int64_t>(p->l2_bytes);
    for (int kernel : {0, 1, 4, 5, 6, 7})
        for (int threads : {128, 256})
            for (int sched = 0; sched < 3; ++sched) {
                if (big && sched == 1) continue;
                const int pf = (kernel >= 6 ? pf_all : 0) | (sched == 0 ? pf_next : 0);
                hs_tuning t{kernel, threads, 1, 0, 0, 0, 0, pf, 0};
                if (sched >= 1) {
                    int occ = 0;
                    // a whitening plan runs its pass on the whitened FP32 copy
                    const bool wh = (sd.flags & HS_FLAG_WHITENING) != 0;
                    const void *fn = fwd1d_kernel(wh ? HS_F32 : sd.dtype, sd.forms & 3, 0, kernel);
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0);
                    if (occ < 1) continue;
                    t.ctas_per_sm = occ;
                    t.dynamic = sched == 2;
                }
                if (validate_tuning(sp, &t) != HS_OK) continue;
                cands.push_back(t);
            }
    for (const hs_tuning &t : cands) {
        sp->tun = t;
        compute_tiles(sp);
        if (upload_tiles(sp) != HS_OK) { result = HS_ERR_CUDA; goto done; }
        const float *wp = (sd.flags & HS_FLAG_WHITENING) ? static_cast<const float *>(w) : nullptr;
        const hs_form_io *ps = (sd.forms & HS_FORM_SIMPLE) ? &fs : nullptr;
        const hs_form_io *pg = (sd.forms & HS_FORM_GREEDY) ? &fg : nullptr;
        float total = 0.f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaMemsetAsync(flush, rep & 0xff, flush_bytes, s);
            cudaEventRecord(e0, s);
            if (enqueue_fwd(sp, x, wp, ps, pg, ws, s, -1, true) != HS_OK) { result = HS_ERR_CUDA; goto done; }
            cudaEventRecord(e1, s);
            if (!cuda_ok(cudaEventSynchronize(e1))) { result = HS_ERR_CUDA; goto done; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) total += ms;
        }
        if (total < best_ms) { best_ms = total; best = t; }
    }
    p->tun = best;
    compute_tiles(p);
    result = upload_tiles(p);
    if (result == HS_OK) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(x);
    cudaFree(tmp);
    cudaFree(w);
    cudaFree(ws);
    cudaFree(outs);
    cudaFree(norm);
    cudaFree(flush);
    hs_plan_destroy(sp);
    return result;
}

// Argument checks shared by hs_run and hs_run_host (device pointers).
hs_status check_run_args(const hs_plan p, const void *spectra, const float *w, const hs_form_io *simple,
                         const hs_form_io *greedy, const void *workspace)
{
    if (!spectra || !aligned(spectra, 16)) return HS_ERR_INVALID_ARG;
    const bool whiten = (p->d.flags & HS_FLAG_WHITENING) != 0;
    if (whiten != (w != nullptr)) return HS_ERR_INVALID_ARG;
    if (w && !aligned(w, 16)) return HS_ERR_INVALID_ARG;
    const bool want_s = (p->d.forms & HS_FORM_SIMPLE) != 0, want_g = (p->d.forms & HS_FORM_GREEDY) != 0;
    if (want_s != (simple != nullptr) || want_g != (greedy != nullptr)) return HS_ERR_INVALID_ARG;
    if (simple) { hs_status st = check_io(p, simple, false); if (st != HS_OK) return st; }
    if (greedy) { hs_status st = check_io(p, greedy, true); if (st != HS_OK) return st; }
    if (p->d.dims == 1 && p->tun.dynamic && (!workspace || !aligned(workspace, 8))) return HS_ERR_INVALID_ARG;
    if (p->d.dims == 2 && workspace && !aligned(workspace, 16)) return HS_ERR_INVALID_ARG;
    return HS_OK;
}

// Host copies of one form's outputs [lo, hi) (and its argmax when `argmax`) on `st`; fields that
// either side leaves NULL are skipped.
hs_status copy_outputs(const hs_plan p, const hs_form_io *dev, const hs_form_io *host, int64_t lo, int64_t hi,
                       bool argmax, cudaStream_t st)
{
    if (!dev || !host || hi <= lo) return HS_OK;
    const size_t n = static_cast<size_t>(hi - lo);
    if (dev->snr && host->snr) HS_CUDA(cudaMemcpyAsync(host->snr + lo, dev->snr + lo, 4 * n, cudaMemcpyDeviceToHost, st));
    if (dev->best_h && host->best_h)
        HS_CUDA(cudaMemcpyAsync(host->best_h + lo, dev->best_h + lo, n, cudaMemcpyDeviceToHost, st));
    if (dev->path && host->path) {
        const size_t pb = static_cast<size_t>(p->path_bytes);
        HS_CUDA(cudaMemcpyAsync(static_cast<unsigned char *>(host->path) + pb * lo,
                                static_cast<const unsigned char *>(dev->path) + pb * lo, pb * n,
                                cudaMemcpyDeviceToHost, st));
    }
    if (argmax && dev->argmax && host->argmax) {
        const int64_t B = p->d.dims == 1 ? p->d.num_spectra : 1;
        HS_CUDA(cudaMemcpyAsync(host->argmax, dev->argmax, sizeof(uint64_t) * B, cudaMemcpyDeviceToHost, st));
    }
    return HS_OK;
}

hs_status ensure_host_streams(hs_plan p)
{
    if (p->h2d) return HS_OK;
    cudaStream_t a = nullptr, b = nullptr;
    HS_CUDA(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
    if (!cuda_ok(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking))) {
        cudaStreamDestroy(a);
        return HS_ERR_CUDA;
    }
    bool ok = cuda_ok(cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming)) &&
              cuda_ok(cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming));
    for (int i = 0; ok && i < kMaxChunks; ++i)
        ok = cuda_ok(cudaEventCreateWithFlags(&p->ev_in[i], cudaEventDisableTiming)) &&
             cuda_ok(cudaEventCreateWithFlags(&p->ev_out[i], cudaEventDisableTiming));
    p->h2d = a;
    p->d2h = b;
    return ok ? HS_OK : HS_ERR_CUDA;
}

}  // namespace

// =========================================================================================
// C ABI
// =========================================================================================
extern "C" {

const char *hs_version(void) { return "1.0.0"; }

const char *hs_last_cuda_error(void) { return g_last_cuda.c_str(); }

const char *hs_status_string(hs_status s)
{
    switch (s) {
    case HS_OK: return "ok";
    case HS_ERR_INVALID_ARG: return "invalid argument";
    case HS_ERR_UNSUPPORTED: return "unsupported";
    case HS_ERR_OOM: return "out of memory";
    case HS_ERR_CUDA: return "CUDA error";
    case HS_ERR_DEVICE_BOUNDS: return "device index out of bounds";
    case HS_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case HS_ERR_NO_DEVICE: return "plan has no device";
    }
    return "unknown status";
}

hs_status hs_norm_exponential(int32_t form, int32_t dims, int32_t H, int32_t mitigation, double mean1,
                              float *mu_out, float *sigma_out)
{
    if (!mu_out || !sigma_out || !(mean1 > 0.0) || !std::isfinite(mean1)) return HS_ERR_INVALID_ARG;
    if (dims == 1) {
        // the optimum over drift paths has no closed-form moments: callers estimate them
        if (form == HS_FORM_OPTIMAL) return HS_ERR_UNSUPPORTED;
        if (H < 1 || H > kMaxH1D || (form != HS_FORM_SIMPLE && form != HS_FORM_GREEDY)) return HS_ERR_INVALID_ARG;
    } else if (dims == 2) {
        if (H < 1 || H > kMaxH2D || form != HS_FORM_GREEDY) return HS_ERR_INVALID_ARG;
    } else {
        return HS_ERR_INVALID_ARG;
    }
    // mean and variance of the maximum of m i.i.d. Exp(1) draws: sum_{k<=m} 1/k, sum 1/k^2
    auto hm = [](int m) { double s = 0; for (int k = 1; k <= m; ++k) s += 1.0 / k; return s; };
    auto hv = [](int m) { double s = 0; for (int k = 1; k <= m; ++k) s += 1.0 / (double(k) * k); return s; };
    for (int h = 1; h <= H; ++h) {
        double mean, var;
        if (dims == 2) {
            mean = hm(9) * h;
            var = hv(9) * h;
        } else if (form == HS_FORM_SIMPLE) {
            mean = h;
            var = h;
        } else if (mitigation) {
            mean = hm(2) * h;
            var = hv(2) * h;
        } else {
            mean = 1.0 + hm(2) * (h - 1);
            var = 1.0 + hv(2) * (h - 1);
        }
        mu_out[h - 1] = static_cast<float>(mean * mean1);
        sigma_out[h - 1] = static_cast<float>(std::sqrt(var) * mean1);
    }
    return HS_OK;
}

hs_status hs_plan_create(hs_plan *out, const hs_desc *desc, int device)
{
    if (!out) return HS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc) return HS_ERR_INVALID_ARG;
    const hs_desc &d = *desc;
    if (d.flags & ~kKnownFlags) return HS_ERR_INVALID_ARG;
    if (d.dtype < HS_F32 || d.dtype > HS_BF16) return HS_ERR_INVALID_ARG;
    hs_plan p = new (std::nothrow) hs_plan_s();
    if (!p) return HS_ERR_OOM;
    p->d = d;
    p->d.lengths = nullptr;
    p->d.offsets = nullptr;
    p->device = device;
    p->no_device = (d.flags & HS_FLAG_NO_DEVICE) != 0;
    if (d.dims == 1) {
        if (d.H < 1 || d.H > kMaxH1D) { delete p; return HS_ERR_INVALID_ARG; }
        if (d.forms < 1 || d.forms > 7) { delete p; return HS_ERR_INVALID_ARG; }
        if (d.num_spectra < 1 || d.num_spectra > (int64_t(1) << 30) || !d.lengths) { delete p; return HS_ERR_INVALID_ARG; }
        const int64_t B = d.num_spectra;
        const int eb = elem_bytes(d.dtype);
        const int64_t al = 16 / eb;
        p->len.assign(d.lengths, d.lengths + B);
        p->in_off.assign(B + 1, 0);
        p->nf.assign(B, 0);
        p->nf_main.assign(B, 0);
        p->fund_off.assign(B + 1, 0);
        int64_t pos = 0;
        for (int64_t s = 0; s < B; ++s) {
            const int64_t n = p->len[s];
            if (n < d.H + 1 || n > 0x7fffffffLL - 64) { delete p; return HS_ERR_INVALID_ARG; }
            int64_t off;
            if (d.offsets) {
                off = d.offsets[s];
                if (off < 0 || off % al) { delete p; return HS_ERR_INVALID_ARG; }
            } else {
                off = (pos + 31) / 32 * 32;
            }
            p->in_off[s] = off;
            pos = off + n;
            p->extent = std::max(p->extent, off + n);
            p->nf_main[s] = (n - 1) / d.H;
            // with the truncated tail every n < N - 1 is a fundamental (its order 1 fits)
            p->nf[s] = (d.flags & HS_FLAG_TRUNCATE_TAIL) ? n - 1 : p->nf_main[s];
            p->fund_off[s + 1] = p->fund_off[s] + p->nf[s];
            p->max_len = std::max(p->max_len, n);
        }
        p->in_off[B] = p->extent;
        if (d.offsets) {   // spectra must not overlap
            std::vector<std::pair<int64_t, int64_t>> iv(B);
            for (int64_t s = 0; s < B; ++s) iv[s] = {p->in_off[s], p->in_off[s] + p->len[s]};
            std::sort(iv.begin(), iv.end());
            for (int64_t s = 1; s < B; ++s)
                if (iv[s].first < iv[s - 1].second) { delete p; return HS_ERR_INVALID_ARG; }
        }
        if (d.flags & HS_FLAG_WHITENING)
            for (int64_t s = 1; s < B; ++s)
                if (p->len[s] != p->len[0]) { delete p; return HS_ERR_INVALID_ARG; }
        p->total_fund = p->fund_off[B];
        p->path_bytes = d.H <= 8 ? 1 : (d.H <= 16 ? 2 : 4);
        p->equal_lengths = std::all_of(p->len.begin(), p->len.end(), [&](int64_t n) { return n == p->len[0]; });
    } else if (d.dims == 2) {
        if (d.H < 1 || d.H > kMaxH2D || d.forms != HS_FORM_GREEDY) { delete p; return HS_ERR_INVALID_ARG; }
        if (d.num_spectra != 1) { delete p; return HS_ERR_INVALID_ARG; }
        if (d.flags & (HS_FLAG_WHITENING | HS_FLAG_PER_SPECTRUM_NORM | HS_FLAG_TRUNCATE_TAIL)) { delete p; return HS_ERR_UNSUPPORTED; }
        if (d.n_freq < 3 || d.n_rows < 3 || d.z0_row < 0 || d.z0_row >= d.n_rows) { delete p; return HS_ERR_INVALID_ARG; }
        if (d.n_freq > (int64_t(1) << 36) || d.n_rows > (int64_t(1) << 20)) { delete p; return HS_ERR_INVALID_ARG; }
        const int64_t H = d.H;
        p->f_lo = 1;
        p->f_hi = (d.n_freq - 1 - H) / H;
        // z with z0 + h z - h >= 0 and z0 + h z + h <= n_rows - 1 for h = 1 and h = H
        auto zok = [&](int64_t z) {
            for (int64_t h : {int64_t(1), H})
                if (d.z0_row + h * z - h < 0 || d.z0_row + h * z + h > d.n_rows - 1) return false;
            return true;
        };
        int64_t zl = 0, zh = 0;
        if (!zok(0)) { delete p; return HS_ERR_INVALID_ARG; }
        while (zok(zl - 1)) --zl;
        while (zok(zh + 1)) ++zh;
        p->z_lo = zl;
        p->z_hi = zh;
        if (p->f_hi < p->f_lo) { delete p; return HS_ERR_INVALID_ARG; }
        p->total_fund = (p->f_hi - p->f_lo + 1) * (p->z_hi - p->z_lo + 1);
        p->extent = d.n_freq * d.n_rows;
        p->path_bytes = 4;
        // z rows fastest: 0.632 ms vs 0.674 ms (f-tiles fastest) on the 201 x 2^21 plane, H = 8; an
        // FP32 plane larger than the device's L2 takes the column sweep instead (below)
        p->tun = hs_tuning{1, 256, 1, 0, 0, 0, 0, 0, 0};
        p->len.assign(1, p->extent);
        p->in_off.assign(2, 0);
        p->in_off[1] = p->extent;
        p->nf.assign(1, p->total_fund);
        p->nf_main.assign(1, p->total_fund);
        p->fund_off = {0, p->total_fund};
        p->max_len = p->extent;
    } else {
        delete p;
        return HS_ERR_INVALID_ARG;
    }
    if (d.dims == 1) p->tun = default_tuning(p);
    compute_tiles(p);
    if (p->no_device) {
        *out = p;
        return HS_OK;
    }
    DeviceGuard guard(device);
    if (!guard.ok) { delete p; return HS_ERR_CUDA; }
    if (!cuda_ok(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, device)) ||
        !cuda_ok(cudaDeviceGetAttribute(&p->l2_bytes, cudaDevAttrL2CacheSize, device))) { delete p; return HS_ERR_CUDA; }
    if (d.dims == 1) {
        // the default launch shape depends on whether the input fits in this device's L2
        p->tun = default_tuning(p);
        compute_tiles(p);
    } else if (d.dtype == HS_F32 && d.H >= 6 && p->extent * 4 >= 8 * static_cast<int64_t>(p->l2_bytes)) {
        // an FP32 plane of 8 L2 sizes or more, summed to 6 orders or more, runs the column sweep where
        // it applies: on 201-row planes, H = 8, it takes 525 us vs 638 us for kernel 1 at 2^21 columns
        // (13 L2 sizes), 294 vs 302 us at 2^20 and 188 vs 135 us at 2^19 (3.3 L2 sizes, where kernel
        // 1's re-reads still mostly hit L2); at 2^21 columns and H = 6 608 vs 615 us, but at H = 4 903
        // vs 654 us and at H = 2 1379 vs 1293 us (fewer orders re-read less, and the domain holds more
        // chains) -- 112-column bands, 1024 threads, chains f < 320 band widths in registers first.
        // 16-bit planes keep kernel 1 (428 us vs 519 us at 2^21, H = 8: half the bytes make kernel
        // 1's re-reads cheaper, while the sweep's cost barely changes).
        const hs_tuning sw{2, 1024, 1, 0, 0, 0, 0, 0, 5};
        const SweepGeom g = sweep_geom(p, sweep_default_wb(d.dtype), sw.threads, 2, kSweepPrefixBands * sw.producers);
        if (g.ok && g.state_bytes + g.sync_bytes <= fwd_workspace_bytes(p)) p->tun = sw;
    }
    const size_t B1 = p->in_off.size();
    if (!cuda_ok(cudaMalloc(&p->d_in_off, sizeof(int64_t) * B1)) ||
        !cuda_ok(cudaMalloc(&p->d_fund_off, sizeof(int64_t) * B1)) ||
        !cuda_ok(cudaMalloc(&p->d_tile_start, sizeof(int64_t) * B1)) ||
        !cuda_ok(cudaMalloc(&p->d_tail_tile_start, sizeof(int64_t) * B1)) ||
        !cuda_ok(cudaMalloc(&p->d_tail1_tile_start, sizeof(int64_t) * B1)) ||
        !cuda_ok(cudaMalloc(&p->d_nf_main, sizeof(int64_t) * (B1 - 1))) ||
        !cuda_ok(cudaMalloc(&p->d_in_len, sizeof(int64_t) * (B1 - 1))) ||
        !cuda_ok(cudaMalloc(&p->d_err, sizeof(int))) ||
        (d.dims == 1 && !cuda_ok(cudaMalloc(&p->d_chunk_tile_start, sizeof(int64_t) * B1 * kMaxChunks)))) {
        free_plan(p);
        return HS_ERR_OOM;
    }
    if (!cuda_ok(cudaMemcpy(p->d_in_off, p->in_off.data(), sizeof(int64_t) * B1, cudaMemcpyHostToDevice)) ||
        !cuda_ok(cudaMemcpy(p->d_fund_off, p->fund_off.data(), sizeof(int64_t) * B1, cudaMemcpyHostToDevice)) ||
        !cuda_ok(cudaMemcpy(p->d_in_len, p->len.data(), sizeof(int64_t) * (B1 - 1), cudaMemcpyHostToDevice)) ||
        !cuda_ok(cudaMemcpy(p->d_nf_main, p->nf_main.data(), sizeof(int64_t) * (B1 - 1), cudaMemcpyHostToDevice)) ||
        !cuda_ok(cudaMemcpy(p->d_tail_tile_start, p->tail_tile_start.data(), sizeof(int64_t) * B1,
                            cudaMemcpyHostToDevice)) ||
        !cuda_ok(cudaMemcpy(p->d_tail1_tile_start, p->tail1_tile_start.data(), sizeof(int64_t) * B1,
                            cudaMemcpyHostToDevice)) ||
        !cuda_ok(cudaMemset(p->d_err, 0, sizeof(int)))) {
        free_plan(p);
        return HS_ERR_CUDA;
    }
    hs_status st = upload_tiles(p);
    if (st == HS_OK && d.dims == 1 && (d.flags & HS_FLAG_AUTOTUNE) && (d.forms & 3)) st = autotune(p);
    if (st != HS_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return HS_OK;
}

hs_status hs_plan_destroy(hs_plan plan)
{
    if (!plan) return HS_ERR_INVALID_ARG;
    free_plan(plan);
    return HS_OK;
}

hs_status hs_plan_fundamentals(hs_plan p, int64_t *counts, int64_t *offsets)
{
    if (!p) return HS_ERR_INVALID_ARG;
    if (counts) std::copy(p->nf.begin(), p->nf.end(), counts);
    if (offsets) std::copy(p->fund_off.begin(), p->fund_off.end(), offsets);
    return HS_OK;
}

hs_status hs_plan_input_offsets(hs_plan p, int64_t *offsets)
{
    if (!p || !offsets) return HS_ERR_INVALID_ARG;
    std::copy(p->in_off.begin(), p->in_off.end(), offsets);
    return HS_OK;
}

hs_status hs_plan_domain_2d(hs_plan p, int64_t *f_lo, int64_t *f_hi, int64_t *z_lo, int64_t *z_hi)
{
    if (!p || p->d.dims != 2) return HS_ERR_INVALID_ARG;
    if (f_lo) *f_lo = p->f_lo;
    if (f_hi) *f_hi = p->f_hi;
    if (z_lo) *z_lo = p->z_lo;
    if (z_hi) *z_hi = p->z_hi;
    return HS_OK;
}

hs_status hs_plan_workspace(hs_plan p, size_t *bytes)
{
    if (!p || !bytes) return HS_ERR_INVALID_ARG;
    *bytes = std::max(fwd_workspace_bytes(p), bwd_workspace_bytes(p));
    return HS_OK;
}

hs_status hs_plan_set_host_chunks(hs_plan p, int32_t chunks)
{
    if (!p || chunks < 0 || chunks > kMaxChunks) return HS_ERR_INVALID_ARG;
    p->host_chunks = chunks;
    if (p->d.dims != 1) return HS_OK;
    make_chunks(p);
    DeviceGuard guard(p->device);
    if (!p->no_device && !guard.ok) return HS_ERR_CUDA;
    return upload_tiles(p);
}

hs_status hs_plan_get_tuning(hs_plan p, hs_tuning *t)
{
    if (!p || !t) return HS_ERR_INVALID_ARG;
    *t = p->tun;
    return HS_OK;
}

hs_status hs_plan_set_tuning(hs_plan p, const hs_tuning *t)
{
    if (!p) return HS_ERR_INVALID_ARG;
    if (p->d.dims == 2) {
        // 2D: kernel 0 = f-tiles fastest, 1 = z rows fastest (256 threads, nothing else);
        // kernel 2 = the column sweep (256 or 512 threads, stage_kb = band width / 16, ctas_per_sm)
        if (!t || t->kernel < 0 || t->kernel > 2 || t->fund_per_thread != 1 || t->dynamic || t->prefetch ||
            t->producers < 0 || t->producers > 64)
            return HS_ERR_INVALID_ARG;
        if (t->kernel < 2 && (t->threads != 256 || t->ctas_per_sm || t->stage_kb || t->stages || t->producers))
            return HS_ERR_INVALID_ARG;
        if (t->kernel == 2) {
            if ((t->threads != 256 && t->threads != 512 && t->threads != 1024) || t->ctas_per_sm < 0 || t->ctas_per_sm > 4 ||
                t->stage_kb < 0 || t->stages < 0 || t->stages == 1 || t->stages > kSweepMaxStages)
                return HS_ERR_INVALID_ARG;
            const int wb = t->stage_kb > 0 ? 16 * t->stage_kb
                                           : sweep_auto_wb(p, t->threads, t->stages > 0 ? t->stages : 2, t->producers);
            const SweepGeom g = sweep_geom(p, wb, t->threads, t->stages > 0 ? t->stages : 2,
                                           kSweepPrefixBands * std::max(1, t->producers));
            if (!g.ok || g.state_bytes + g.sync_bytes > fwd_workspace_bytes(p)) return HS_ERR_UNSUPPORTED;
        }
        std::lock_guard<std::mutex> lk(p->mu);
        p->tun = *t;
        p->gvalid = false;
        return HS_OK;
    }
    if (p->d.dims != 1) return HS_ERR_UNSUPPORTED;
    hs_status st = validate_tuning(p, t);
    if (st != HS_OK) return st;
    std::lock_guard<std::mutex> lk(p->mu);
    p->tun = *t;
    compute_tiles(p);
    p->gvalid = false;
    if (p->no_device) return HS_OK;
    DeviceGuard guard(p->device);
    if (!guard.ok) return HS_ERR_CUDA;
    return upload_tiles(p);
}

hs_status hs_run(hs_plan p, const void *spectra, const float *w, const hs_form_io *simple,
                 const hs_form_io *greedy, void *workspace, void *stream)
{
    if (!p) return HS_ERR_INVALID_ARG;
    if (p->no_device) return HS_ERR_NO_DEVICE;
    const hs_status vs = check_run_args(p, spectra, w, simple, greedy, workspace);
    if (vs != HS_OK) return vs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DeviceGuard guard(p->device);
    if (!guard.ok) return HS_ERR_CUDA;
    if (!(p->d.flags & HS_FLAG_GRAPH)) return enqueue_fwd(p, spectra, w, simple, greedy, workspace, st, -1, true);

    // graph replay: capture once per argument set on a private stream, launch on `st`
    std::lock_guard<std::mutex> lk(p->mu);
    GraphKey k{};
    std::memset(&k, 0, sizeof(k));
    k.spectra = spectra;
    k.w = w;
    k.ws = workspace;
    if (simple) k.s = *simple;
    if (greedy) k.g = *greedy;
    if (!(p->gvalid && k == p->gkey)) {
        if (!p->cap && !cuda_ok(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking)))
            return enqueue_fwd(p, spectra, w, simple, greedy, workspace, st, -1, true);
        cudaGraph_t g = nullptr;
        bool ok = cuda_ok(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
        if (ok) {
            hs_status es = enqueue_fwd(p, spectra, w, simple, greedy, workspace, p->cap, -1, true);
            ok = cuda_ok(cudaStreamEndCapture(p->cap, &g)) && es == HS_OK && g;
        }
        if (ok) {
            if (p->gexec) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(p->gexec, g, &info) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(p->gexec);
                    p->gexec = nullptr;
                }
            }
            if (!p->gexec && !cuda_ok(cudaGraphInstantiate(&p->gexec, g, 0))) {
                p->gexec = nullptr;
                ok = false;
            }
        }
        if (g) cudaGraphDestroy(g);
        if (!ok) {   // capture failed: fall back to a direct launch
            cudaGetLastError();
            p->gvalid = false;
            return enqueue_fwd(p, spectra, w, simple, greedy, workspace, st, -1, true);
        }
        p->gkey = k;
        p->gvalid = true;
    }
    HS_CUDA(cudaGraphLaunch(p->gexec, st));
    return HS_OK;
}

hs_status hs_run_host(hs_plan p, const void *host_spectra, void *spectra, const float *w, const hs_form_io *simple,
                      const hs_form_io *greedy, const hs_form_io *host_simple, const hs_form_io *host_greedy,
                      void *workspace, void *stream)
{
    if (!p) return HS_ERR_INVALID_ARG;
    if (p->no_device) return HS_ERR_NO_DEVICE;
    if (!host_spectra || host_spectra == spectra) return HS_ERR_INVALID_ARG;
    const hs_status vs = check_run_args(p, spectra, w, simple, greedy, workspace);
    if (vs != HS_OK) return vs;
    if ((host_simple && !simple) || (host_greedy && !greedy)) return HS_ERR_INVALID_ARG;
    if (host_simple && host_simple->path) return HS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DeviceGuard guard(p->device);
    if (!guard.ok) return HS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(p->mu);   // the plan's copy streams and events
    hs_status es = ensure_host_streams(p);
    if (es != HS_OK) return es;
    const int64_t eb = elem_bytes(p->d.dtype);
    const unsigned char *hsrc = static_cast<const unsigned char *>(host_spectra);
    unsigned char *ddst = static_cast<unsigned char *>(spectra);
    // the copies wait for the work already on `stream` (it may still read the device buffer)
    HS_CUDA(cudaEventRecord(p->ev_start, st));
    HS_CUDA(cudaStreamWaitEvent(p->h2d, p->ev_start, 0));
    HS_CUDA(cudaStreamWaitEvent(p->d2h, p->ev_start, 0));
    const bool host_out = host_simple || host_greedy;
    const int K = p->d.dims == 1 ? static_cast<int>(p->chunks.size()) : 1;
    if (K <= 1) {
        HS_CUDA(cudaMemcpyAsync(ddst, hsrc, static_cast<size_t>(p->extent * eb), cudaMemcpyHostToDevice, p->h2d));
        HS_CUDA(cudaEventRecord(p->ev_in[0], p->h2d));
        HS_CUDA(cudaStreamWaitEvent(st, p->ev_in[0], 0));
        es = enqueue_fwd(p, spectra, w, simple, greedy, workspace, st);
        if (es != HS_OK) return es;
        if (host_out) {
            HS_CUDA(cudaEventRecord(p->ev_out[0], st));
            HS_CUDA(cudaStreamWaitEvent(p->d2h, p->ev_out[0], 0));
            es = copy_outputs(p, simple, host_simple, 0, p->total_fund, true, p->d2h);
            if (es == HS_OK) es = copy_outputs(p, greedy, host_greedy, 0, p->total_fund, true, p->d2h);
            if (es != HS_OK) return es;
        }
    } else {
        const int64_t B = p->d.num_spectra;
        if (simple && simple->argmax) HS_CUDA(cudaMemsetAsync(simple->argmax, 0, sizeof(uint64_t) * B, st));
        if (greedy && greedy->argmax) HS_CUDA(cudaMemsetAsync(greedy->argmax, 0, sizeof(uint64_t) * B, st));
        for (int c = 0; c < K; ++c) {
            const auto &ch = p->chunks[c];
            if (ch.in_hi > ch.in_lo)
                HS_CUDA(cudaMemcpyAsync(ddst + ch.in_lo * eb, hsrc + ch.in_lo * eb,
                                        static_cast<size_t>((ch.in_hi - ch.in_lo) * eb), cudaMemcpyHostToDevice,
                                        p->h2d));
            HS_CUDA(cudaEventRecord(p->ev_in[c], p->h2d));
            HS_CUDA(cudaStreamWaitEvent(st, p->ev_in[c], 0));
            es = enqueue_fwd(p, spectra, w, simple, greedy, workspace, st, c);
            if (es != HS_OK) return es;
            const bool lastc = c + 1 == K;
            if (host_out && (p->chunk_out || lastc)) {
                HS_CUDA(cudaEventRecord(p->ev_out[c], st));
                HS_CUDA(cudaStreamWaitEvent(p->d2h, p->ev_out[c], 0));
                const int64_t lo = p->chunk_out ? ch.out_lo : 0, hi = p->chunk_out ? ch.out_hi : p->total_fund;
                es = copy_outputs(p, simple, host_simple, lo, hi, lastc, p->d2h);
                if (es == HS_OK) es = copy_outputs(p, greedy, host_greedy, lo, hi, lastc, p->d2h);
                if (es != HS_OK) return es;
            }
        }
    }
    // `stream` continues once the last copy in either direction has been issued before it
    HS_CUDA(cudaEventRecord(p->ev_done, p->d2h));
    HS_CUDA(cudaStreamWaitEvent(st, p->ev_done, 0));
    return HS_OK;
}

hs_status hs_run_optimal(hs_plan p, const void *spectra, const float *w, const hs_form_io *optimal, void *stream)
{
    if (!p) return HS_ERR_INVALID_ARG;
    if (p->no_device) return HS_ERR_NO_DEVICE;
    if (p->d.dims != 1 || !(p->d.forms & HS_FORM_OPTIMAL)) return HS_ERR_INVALID_ARG;
    if (!spectra || !aligned(spectra, 16)) return HS_ERR_INVALID_ARG;
    const bool whiten = (p->d.flags & HS_FLAG_WHITENING) != 0;
    if (whiten != (w != nullptr)) return HS_ERR_INVALID_ARG;
    if (w && !aligned(w, 16)) return HS_ERR_INVALID_ARG;
    {
        hs_status cs = check_io(p, optimal, true);
        if (cs != HS_OK) return cs;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DeviceGuard guard(p->device);
    if (!guard.ok) return HS_ERR_CUDA;
    const int64_t B = p->d.num_spectra;
    if (optimal->argmax) HS_CUDA(cudaMemsetAsync(optimal->argmax, 0, sizeof(uint64_t) * B, st));
    Fwd1DArgs a{};
    a.x = spectra;
    a.w = w;
    a.in_off = p->d_in_off;
    a.fund_off = p->d_fund_off;
    a.in_len = p->d_in_len;
    a.nf_main = p->d_nf_main;
    a.B = static_cast<int32_t>(B);
    a.H = p->d.H;
    a.mitigation = (p->d.flags & HS_FLAG_NO_MITIGATION) ? 0 : 1;
    a.per_spectrum_norm = (p->d.flags & HS_FLAG_PER_SPECTRUM_NORM) ? 1 : 0;
    a.path_bytes = p->path_bytes;
    a.checked = (p->d.flags & HS_FLAG_CHECKED) ? 1 : 0;
    a.err = p->d_err;
    FormArgs o = to_form_args(optimal);
    // one warp per fundamental; each warp takes a contiguous run of fundamentals
    const int threads = 256, wpc = threads / 32;
    int64_t F = p->total_fund;
    const void *fn = fwd1d_opt_kernel(p->d.dtype, whiten ? 1 : 0, p->d.H, (p->d.flags & HS_FLAG_TRUNCATE_TAIL) ? 1 : 0);
    if (!fn) return HS_ERR_UNSUPPORTED;
    int occ = 0;
    HS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0));
    // one wave of resident CTAs
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>((F + wpc - 1) / wpc,
                                                                static_cast<int64_t>(p->sms) * std::max(occ, 1)));
    int64_t chunk = (F + ctas * wpc - 1) / (ctas * wpc);
    void *args[] = {&a, &o, &F, &chunk};
    HS_CUDA(cudaLaunchKernel(fn, dim3(static_cast<unsigned>(ctas)), dim3(threads), args, 0, st));
    return HS_OK;
}

hs_status hs_backward(hs_plan p, int32_t form, const float *grad_snr, const hs_form_io *fwd,
                      const void *spectra, const float *w, float *grad_in, float *grad_w,
                      void *workspace, void *stream)
{
    if (!p) return HS_ERR_INVALID_ARG;
    if (p->no_device) return HS_ERR_NO_DEVICE;
    if (p->d.dims != 1) return HS_ERR_UNSUPPORTED;
    if (form != HS_FORM_SIMPLE && form != HS_FORM_GREEDY && form != HS_FORM_OPTIMAL) return HS_ERR_INVALID_ARG;
    if (!(p->d.forms & form)) return HS_ERR_INVALID_ARG;
    if (!grad_snr || !fwd || !fwd->best_h || !fwd->sigma) return HS_ERR_INVALID_ARG;
    if (form != HS_FORM_SIMPLE && !fwd->path) return HS_ERR_INVALID_ARG;
    // the optimal form's bins follow its recorded drift path exactly as the greedy form's do
    const int kform = form == HS_FORM_SIMPLE ? HS_FORM_SIMPLE : HS_FORM_GREEDY;
    if (!aligned(grad_snr, 4) || !aligned(fwd->sigma, 4)) return HS_ERR_INVALID_ARG;
    if (fwd->path && !aligned(fwd->path, p->path_bytes)) return HS_ERR_INVALID_ARG;
    const bool whiten = (p->d.flags & HS_FLAG_WHITENING) != 0;
    if (whiten != (w != nullptr)) return HS_ERR_INVALID_ARG;
    if (grad_w && !whiten) return HS_ERR_INVALID_ARG;
    if (grad_w && (!spectra || !aligned(spectra, 16))) return HS_ERR_INVALID_ARG;
    if (!grad_in && !grad_w) return HS_OK;
    if ((grad_in && !aligned(grad_in, 4)) || (grad_w && !aligned(grad_w, 4))) return HS_ERR_INVALID_ARG;
    const int64_t B = p->d.num_spectra;
    Bwd1DArgs a{};
    a.form = kform;
    a.H = p->d.H;
    a.B = static_cast<int32_t>(B);
    a.path_bytes = p->path_bytes;
    a.grad_snr = grad_snr;
    a.best_h = fwd->best_h;
    a.path = fwd->path;
    a.sigma = fwd->sigma;
    a.per_spectrum_norm = (p->d.flags & HS_FLAG_PER_SPECTRUM_NORM) ? 1 : 0;
    a.p = spectra;
    a.dtype = p->d.dtype;
    a.w = w;
    a.in_off = p->d_in_off;
    a.in_len = p->d_in_len;
    a.fund_off = p->d_fund_off;
    a.grad_in = grad_in;
    a.grad_w = grad_w;
    a.n_common = p->len[0];
    a.block_bins = kBwdBlockBins;
    a.group = 1;
    a.dw_partial = nullptr;
    // candidates of a block: sum over k of (floor((L-1)/k) + 2) (greedy), bounded generously
    int max_cand = 0;
    for (int k = 1; k <= p->d.H; ++k) max_cand += (kBwdBlockBins - 1) / k + 3;
    a.max_cand = max_cand;
    a.err = p->d_err;
    int64_t gx;
    int gy;
    if (grad_w) {
        gx = (p->len[0] + kBwdBlockBins - 1) / kBwdBlockBins;
        gy = bwd_groups(p);
        a.group = static_cast<int32_t>((B + gy - 1) / gy);
        gy = static_cast<int>((B + a.group - 1) / a.group);
        if (gy > 1) {
            if (!workspace || !aligned(workspace, 16)) return HS_ERR_INVALID_ARG;
            a.dw_partial = static_cast<float *>(workspace);
        }
    } else {
        gx = (p->max_len + kBwdBlockBins - 1) / kBwdBlockBins;
        if (B > 65535) return HS_ERR_UNSUPPORTED;
        gy = static_cast<int>(B);
    }
    if (gx > 0x7fffffff) return HS_ERR_UNSUPPORTED;
    a.blocks_per_spectrum = gx;
    if (workspace && !aligned(workspace, 16)) return HS_ERR_INVALID_ARG;
    const void *fn = bwd1d_kernel(kform, p->d.dtype, whiten ? 1 : 0);
    if (!fn) return HS_ERR_UNSUPPORTED;
    DeviceGuard guard(p->device);
    if (!guard.ok) return HS_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (workspace) {
        // with a workspace, mark the bin blocks that receive contributions; the rest skip staging
        a.nblk = bwd_nblk(p);
        uint8_t *wsb = static_cast<uint8_t *>(workspace) + bwd_partial_bytes(p);
        a.active = wsb;
        a.nz_count = reinterpret_cast<int *>(wsb + bwd_flag_bytes(p));
        a.nz_list = a.nz_count + (B + 63) / 64 * 64;
        // flags and counts are contiguous: one memset clears both
        HS_CUDA(cudaMemsetAsync(a.active, 0, bwd_flag_bytes(p) + static_cast<size_t>(B) * 4, st));
        int64_t F = p->total_fund;
        void *margs[] = {&a, &F};
        const unsigned mgrid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((F + 255) / 256, 16 * p->sms)));
        HS_CUDA(cudaLaunchKernel(bwd_mark_kernel(kform), dim3(mgrid), dim3(256), margs, 0, st));
    }
    void *args[] = {&a};
    const size_t smem = kBwdBlockBins * sizeof(long long) + max_cand * (sizeof(float) + sizeof(int16_t));
    {
        hs_status es = ensure_bwd_smem(fn, smem);
        if (es != HS_OK) return es;
    }
    HS_CUDA(cudaLaunchKernel(fn, dim3(static_cast<unsigned>(gx), gy), dim3(kBwdThreads), args, smem, st));
    if (grad_w && gy > 1) {
        const float *part = a.dw_partial;
        int groups = gy;
        int64_t n = p->len[0];
        float *gw = grad_w;
        void *rargs[] = {&part, &groups, &n, &gw};
        const unsigned rgrid = static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 8 * p->sms));
        HS_CUDA(cudaLaunchKernel(bwd_dw_reduce_kernel(), dim3(rgrid), dim3(256), rargs, 0, st));
    }
    return HS_OK;
}

hs_status hs_selftest_timeout(hs_plan p, uint32_t limit_us, void *stream)
{
    if (!p) return HS_ERR_INVALID_ARG;
    if (p->no_device) return HS_ERR_NO_DEVICE;
    if (limit_us < 1 || limit_us > 1000000) return HS_ERR_INVALID_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return HS_ERR_CUDA;
    unsigned long long limit_ns = 1000ull * limit_us;
    void *args[] = {&p->d_err, &limit_ns};
    HS_CUDA(cudaLaunchKernel(wait_selftest_kernel(), dim3(1), dim3(32), args, 0, static_cast<cudaStream_t>(stream)));
    return HS_OK;
}

hs_status hs_check_device_error(hs_plan p, void *stream)
{
    if (!p) return HS_ERR_INVALID_ARG;
    if (p->no_device) return HS_ERR_NO_DEVICE;
    DeviceGuard guard(p->device);
    if (!guard.ok) return HS_ERR_CUDA;
    HS_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int e = 0;
    HS_CUDA(cudaMemcpy(&e, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != kErrNone) HS_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
    if (e == kErrBounds) return HS_ERR_DEVICE_BOUNDS;
    if (e == kErrTimeout) return HS_ERR_DEVICE_TIMEOUT;
    return HS_OK;
}

// -----------------------------------------------------------------------------------------
// Forward pass without any caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they run the harmonic sum:
// plug-ins whose host framework owns every allocation, real-time pipelines that forbid
// allocation after start-up, and code that only receives input and output pointers.  For
// them the scratch the forward needs (the tile counter of the dynamic schedule) lives in
// the fixed array below, which the library's module holds on every GPU that loads it until
// the process exits.  In host code `g_fixed_scratch` names a host-side stand-in, not a device
// address, so every call looks up its device address (cudaGetSymbolAddress, with the plan's
// device current) and passes that to the kernels.  The lookup is not cached: a device reset or
// a re-created primary context reloads the module at a new address, and a cached address would
// then point at freed memory.
// -----------------------------------------------------------------------------------------
constexpr size_t kFixedScratchBytes = 4096;
static __device__ __align__(256) unsigned char g_fixed_scratch[kFixedScratchBytes];

namespace {
// Device address of g_fixed_scratch in the current context (the caller makes the device current).
hs_status fixed_scratch_ptr(void **out)
{
    void *ptr = nullptr;
    HS_CUDA(cudaGetSymbolAddress(&ptr, g_fixed_scratch));
    if (!ptr) return HS_ERR_CUDA;
    *out = ptr;
    return HS_OK;
}
}  // namespace

hs_status hs_run_fixed_scratch(hs_plan p, const void *spectra, const float *w, const hs_form_io *simple,
                               const hs_form_io *greedy, void *stream)
{
    if (!p) return HS_ERR_INVALID_ARG;
    if (p->no_device) return HS_ERR_NO_DEVICE;
    // more scratch than the array (1D); a 2D plan runs without workspace (kernel 2 then runs as 1)
    // (a whitening plan runs here without its whitened copy: the pass multiplies as it loads)
    if (p->d.dims == 1 && kWorkspaceBytes > kFixedScratchBytes) return HS_ERR_UNSUPPORTED;
    if (!spectra || !aligned(spectra, 16)) return HS_ERR_INVALID_ARG;
    const bool whiten = (p->d.flags & HS_FLAG_WHITENING) != 0;
    if (whiten != (w != nullptr)) return HS_ERR_INVALID_ARG;
    if (w && !aligned(w, 16)) return HS_ERR_INVALID_ARG;
    const bool want_s = (p->d.forms & HS_FORM_SIMPLE) != 0, want_g = (p->d.forms & HS_FORM_GREEDY) != 0;
    if (want_s != (simple != nullptr) || want_g != (greedy != nullptr)) return HS_ERR_INVALID_ARG;
    if (simple) { hs_status st = check_io(p, simple, false); if (st != HS_OK) return st; }
    if (greedy) { hs_status st = check_io(p, greedy, true); if (st != HS_OK) return st; }
    DeviceGuard guard(p->device);
    if (!guard.ok) return HS_ERR_CUDA;
    void *scratch = nullptr;
    hs_status st = fixed_scratch_ptr(&scratch);
    if (st != HS_OK) return st;
    std::lock_guard<std::mutex> lk(p->mu);
    return enqueue_fwd(p, spectra, w, simple, greedy, p->d.dims == 1 ? scratch : nullptr,
                       static_cast<cudaStream_t>(stream));
}

}  // extern "C"
