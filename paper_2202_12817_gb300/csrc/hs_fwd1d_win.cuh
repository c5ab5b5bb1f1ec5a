// Window-staged 1D forward (kernel 2).
//
// For a tile of T consecutive fundamentals [n0, n0 + T) the order-h window
// [h n0, h (n0 + T - 1) + h] holds every bin that any fundamental of the tile can read at that
// order: the simple form reads h n (Eq. 3), the greedy form h n + d and h n + d + 1 with
// d <= h - 1 (Eq. 5, Algorithm 2).  Each window is copied from global memory into shared
// memory with one 1D bulk copy (cp.async.bulk, the TMA engine), so the L2 -> SM traffic is
// fully coalesced (a strided / drift-dependent gather would pay one 32-byte sector per 4-byte
// value), and the greedy comparison chain runs on shared-memory latency instead of L2 latency.
//
// Roles: warp T/32 is the producer (one elected lane issues the bulk copies); warps 0..T/32-1
// are consumers, one fundamental per thread.  The orders of a tile are packed into phases,
// each filling one buffer of an nbuf-deep ring; `full[b]` completes when a phase's bytes
// land (expect-tx), `empty[b]` when every consumer warp is done with the buffer.  Every wait
// is bounded (kWaitNs of global time); a timed-out wait sets the device error word, raises an
// abort flag and the CTA winds down after draining its own copies in flight.
#pragma once

#include "hs_fwd1d.cuh"

namespace hs {

constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s
constexpr int kMaxBuf = 4;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the completion of phase `parity` of `bar`; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void consumer_sync(int nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

template <typename T>
__device__ __forceinline__ float sm_ld(const T *w, int i);
template <>
__device__ __forceinline__ float sm_ld<float>(const float *w, int i) { return w[i]; }
template <>
__device__ __forceinline__ float sm_ld<__half>(const __half *w, int i) { return __half2float(w[i]); }
template <>
__device__ __forceinline__ float sm_ld<__nv_bfloat16>(const __nv_bfloat16 *w, int i)
{
    return __bfloat162float(w[i]);
}

// consumer-only block max of a 64-bit key, then one atomicMax
__device__ __forceinline__ void consumer_argmax(unsigned long long key, unsigned long long *dst,
                                                unsigned long long *scratch, int nthreads)
{
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
        key = k2 > key ? k2 : key;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) scratch[warp] = key;
    consumer_sync(nthreads);
    if (warp == 0) {
        const int nw = nthreads >> 5;
        key = lane < nw ? scratch[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
            key = k2 > key ? k2 : key;
        }
        if (lane == 0 && key != 0ull) atomicMax(dst, key);
    }
    consumer_sync(nthreads);
}

template <typename T, int FORMS>
__global__ void __launch_bounds__(288) k_fwd1d_win(const Fwd1DArgs a, const WinPlan wp)
{
    extern __shared__ __align__(128) unsigned char win_smem[];
    __shared__ NormSmem nm;
    __shared__ unsigned long long red[32];
    __shared__ __align__(8) uint64_t full[kMaxBuf], empty[kMaxBuf];
    __shared__ volatile int s_abort;
    constexpr bool kS = (FORMS & HS_FORM_SIMPLE) != 0;
    constexpr bool kG = (FORMS & HS_FORM_GREEDY) != 0;
    constexpr int A = 16 / static_cast<int>(sizeof(T));   // elements per 16 bytes
    const int Tn = wp.T;
    const int ncw = Tn >> 5;                               // consumer warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int H = a.H;

    if (threadIdx.x == 0) {
        for (int b = 0; b < wp.nbuf; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], ncw);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ------------------------------------------------------------------ producer
    if (warp == ncw) {
        if (lane != 0) return;
        uint32_t q = 0;
        int issued_u[kMaxBuf];
        for (int b = 0; b < kMaxBuf; ++b) issued_u[b] = -1;
        bool ok = true;
        for (int64_t tile = blockIdx.x; ok && tile < a.total_tiles; tile += gridDim.x) {
            const int s = tile_spectrum(a.tile_start, a.B, tile);
            const int64_t fbase = __ldg(a.fund_off + s);
            const int64_t nf = __ldg(a.fund_off + s + 1) - fbase;
            const int64_t n0 = (tile - __ldg(a.tile_start + s)) * Tn;
            const int64_t n_last = (n0 + Tn < nf ? n0 + Tn : nf) - 1;
            const int64_t base = __ldg(a.in_off + s);
            const int64_t avail = wp.extent - base;           // readable elements from x
            const T *x = static_cast<const T *>(a.x) + base;
            for (int p = 0; p < wp.nphase; ++p, ++q) {
                const int b = static_cast<int>(q % wp.nbuf);
                const int u = static_cast<int>(q / wp.nbuf);
                if (u > 0 && !mbar_wait(&empty[b], (u - 1) & 1)) {
                    set_error(a.err, kErrTimeout);
                    s_abort = 1;
                    ok = false;
                    break;
                }
                if (s_abort) { ok = false; break; }
                unsigned char *buf = win_smem + static_cast<size_t>(b) * wp.buf_bytes;
                uint32_t bytes = 0;
                for (int h = wp.phase_h0[p]; h < wp.phase_h0[p + 1]; ++h) {
                    const int64_t g0 = static_cast<int64_t>(h) * n0;
                    const int64_t g1 = static_cast<int64_t>(h) * n_last + h + 1;   // exclusive
                    const int64_t g0a = g0 & ~static_cast<int64_t>(A - 1);
                    const int64_t g1u = (g1 + A - 1) & ~static_cast<int64_t>(A - 1);
                    const int64_t gc = g1u <= avail ? g1u : (g1 & ~static_cast<int64_t>(A - 1));
                    T *dst = reinterpret_cast<T *>(buf + wp.off[h - 1]);
                    if (gc > g0a) {
                        const uint32_t nb = static_cast<uint32_t>((gc - g0a) * static_cast<int64_t>(sizeof(T)));
                        bulk_g2s(dst, x + g0a, nb, &full[b]);
                        bytes += nb;
                    }
                    for (int64_t j = (gc > g0a ? gc : g0a); j < g1; ++j) dst[j - g0a] = x[j];   // unaligned tail
                }
                mbar_arrive_expect_tx(&full[b], bytes);
                issued_u[b] = u;
            }
        }
        if (!ok) {
            // drain: wait (bounded) until every copy this CTA issued has landed
            for (int b = 0; b < wp.nbuf; ++b)
                if (issued_u[b] >= 0) mbar_wait(&full[b], issued_u[b] & 1);
        }
        return;
    }

    // ------------------------------------------------------------------ consumers
    const int t = threadIdx.x;
    uint32_t q = 0;
    int loaded_spec = -1;
    for (int64_t tile = blockIdx.x; tile < a.total_tiles; tile += gridDim.x) {
        const int s = tile_spectrum(a.tile_start, a.B, tile);
        if (s != loaded_spec) {
            consumer_sync(Tn);
            const int64_t no = a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0;
            if (kS) load_norm(nm, 0, a.s.mu + no, a.s.sigma + no, H);
            if (kG) load_norm(nm, 1, a.g.mu + no, a.g.sigma + no, H);
            consumer_sync(Tn);
            loaded_spec = s;
        }
        const int64_t fbase = __ldg(a.fund_off + s);
        const int64_t nf = __ldg(a.fund_off + s + 1) - fbase;
        const int64_t n0 = (tile - __ldg(a.tile_start + s)) * Tn;
        const int64_t n = n0 + t;
        const bool valid = n < nf;
        RunMax ms{0.f, 1}, mg{0.f, 1};
        float ss = 0.f, sg = 0.f;
        int d = 0;
        uint32_t bits = 0;
        for (int p = 0; p < wp.nphase; ++p, ++q) {
            const int b = static_cast<int>(q % wp.nbuf);
            const int u = static_cast<int>(q / wp.nbuf);
            // after an abort, waits are skipped (the data is garbage, the error word is set) so
            // that every consumer still reaches the same named barriers
            if (!s_abort && !mbar_wait(&full[b], u & 1)) {
                set_error(a.err, kErrTimeout);
                s_abort = 1;
            }
            const unsigned char *buf = win_smem + static_cast<size_t>(b) * wp.buf_bytes;
            if (valid) {
                for (int h = wp.phase_h0[p]; h < wp.phase_h0[p + 1]; ++h) {
                    const T *w = reinterpret_cast<const T *>(buf + wp.off[h - 1]);
                    const int64_t g0 = static_cast<int64_t>(h) * n0;
                    const int e = h * t + static_cast<int>(g0 - (g0 & ~static_cast<int64_t>(A - 1)));
                    if (h == 1) {
                        const float x0 = sm_ld<T>(w, e);
                        ss = x0;
                        sg = x0;
                        if (kG && a.mitigation) {
                            const float x1 = sm_ld<T>(w, e + 1);
                            if (x1 > x0) { d = 1; sg = x1; bits = 1u; }
                        }
                        if (kS) ms.first(fmaf(ss, nm.rs[0][0], -nm.murs[0][0]));
                        if (kG) mg.first(fmaf(sg, nm.rs[1][0], -nm.murs[1][0]));
                    } else {
                        if (kS) {
                            ss += sm_ld<T>(w, e);
                            ms.step(fmaf(ss, nm.rs[0][h - 1], -nm.murs[0][h - 1]), h);
                        }
                        if (kG) {
                            const float va = sm_ld<T>(w, e + d);
                            const float vb = sm_ld<T>(w, e + d + 1);
                            const bool inc = vb > va;
                            sg += inc ? vb : va;
                            d += inc;
                            bits |= static_cast<uint32_t>(inc) << (h - 1);
                            mg.step(fmaf(sg, nm.rs[1][h - 1], -nm.murs[1][h - 1]), h);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[b]);
        }
        if (valid && !s_abort) {
            const int64_t o = fbase + n;
            if (kS) {
                a.s.snr[o] = ms.best;
                a.s.best_h[o] = static_cast<uint8_t>(ms.bh);
            }
            if (kG) {
                a.g.snr[o] = mg.best;
                a.g.best_h[o] = static_cast<uint8_t>(mg.bh);
                if (a.g.path) store_path(a.g.path, a.path_bytes, o, bits);
            }
        }
        if (kS && a.s.argmax) consumer_argmax(valid ? argmax_key(ms.best, n) : 0ull, a.s.argmax + s, red, Tn);
        if (kG && a.g.argmax) consumer_argmax(valid ? argmax_key(mg.best, n) : 0ull, a.g.argmax + s, red, Tn);
    }
}

template <typename T>
static const void *fwd1d_win_kernel_for(int forms)
{
    switch (forms) {
    case 1: return reinterpret_cast<const void *>(&k_fwd1d_win<T, 1>);
    case 2: return reinterpret_cast<const void *>(&k_fwd1d_win<T, 2>);
    case 3: return reinterpret_cast<const void *>(&k_fwd1d_win<T, 3>);
    }
    return nullptr;
}

}  // namespace hs
