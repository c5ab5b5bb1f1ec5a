// Window-staged 1D forward (kernel 2).
//
// For a tile of T consecutive fundamentals [n0, n0 + T) the order-h window
// [h n0, h (n0 + T - 1) + h] holds every bin that any fundamental of the tile can read at that
// order: the simple form reads h n (Eq. 3), the greedy form h n + d and h n + d + 1 with
// d <= h - 1 (Eq. 5, Algorithm 2).  Each window is copied from global memory into shared
// memory with one 1D bulk copy (cp.async.bulk, the TMA engine), so the L2 -> SM traffic is
// fully coalesced (a strided / drift-dependent gather pays one 32-byte sector per 4-byte
// value), and the greedy comparison chain runs on shared-memory latency instead of L2 latency.
//
// A CTA walks the sequence j = 0, 1, 2, ... of (tile k, order h) pairs, j = k H + h - 1, through
// a ring of `nslot` slots: order j lives in slot j % nslot.  Bulk copies issued by one warp
// complete one after another (~0.3 us each on this part), so `nprod` producer warps share the
// issuing -- order j is issued by producer warp j % nprod -- to keep several copies in flight.
// T consumer threads (one fundamental each) take the orders in sequence.  `full[i]` completes
// when slot i's bytes land (expect-tx), `empty[i]` when every consumer warp is done with it.
// Every wait is bounded (kWaitNs of global time); a timed-out wait sets the device error word
// and raises an abort flag, after which nobody waits any more and producers drain their own
// copies in flight before returning.
#pragma once

#include "hs_fwd1d.cuh"

namespace hs {

constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s
constexpr int kMaxSlot = 16;

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

// Wait for the completion of phase `parity` of `bar`; false after limit_ns (default kWaitNs).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns = kWaitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
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

__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
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
        if (lane == 0 && key != 0ull) {
            wait_prior_grid();
            argmax_update(dst, key);
        }
    }
    consumer_sync(nthreads);
}

template <typename T, int FORMS>
__global__ void __launch_bounds__(640) k_fwd1d_win(const Fwd1DArgs a, const WinPlan wp)
{
    extern __shared__ __align__(128) unsigned char win_smem[];
    __shared__ unsigned long long red[32];
    __shared__ __align__(8) uint64_t full[kMaxSlot], empty[kMaxSlot];
    __shared__ float2 nrm[2][kMaxH1D];      // (1/sigma_h, mu_h/sigma_h) per form
    __shared__ volatile int s_abort;
    constexpr bool kS = (FORMS & HS_FORM_SIMPLE) != 0;
    constexpr bool kG = (FORMS & HS_FORM_GREEDY) != 0;
    constexpr int A = 16 / static_cast<int>(sizeof(T));   // elements per 16 bytes
    const int Tn = wp.T;
    const int ncw = Tn >> 5;                               // consumer warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int H = a.H;
    const int R = wp.nslot;

    if (threadIdx.x == 0) {
        for (int i = 0; i < R; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], ncw);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // tiles of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int64_t my_tiles = a.total_tiles > blockIdx.x
                                 ? (a.total_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const int64_t total_j = my_tiles * H;

    // ------------------------------------------------------------------ producers
    if (warp >= ncw) {
        const int pw = warp - ncw;
        if (lane != 0) return;
        if (pw == 0 && wp.pf_chunk > 0) {
            // the whole input fits comfortably in L2: bring this CTA's share in ahead of the windows
            const int64_t total = wp.extent * static_cast<int64_t>(sizeof(T));
            int64_t lo = static_cast<int64_t>(blockIdx.x) * wp.pf_chunk;
            const int64_t hi = lo + wp.pf_chunk < total ? lo + wp.pf_chunk : total;
            const unsigned char *src = static_cast<const unsigned char *>(a.x);
            for (; lo + 16 <= hi; lo += 65536) {
                const int64_t nb = (hi - lo < 65536 ? hi - lo : 65536) & ~static_cast<int64_t>(15);
                bulk_prefetch_l2(src + lo, static_cast<uint32_t>(nb));
            }
        }
        // this warp issues orders j = pw, pw + P, ...; (k, h) = (j / H, j % H + 1) and
        // (slot, use) = (j % R, j / R) are stepped incrementally (no divisions in the loop)
        const int P = wp.nprod;
        int64_t k = 0;
        int h = pw + 1;
        while (h > H) { h -= H; ++k; }
        int slot = pw % R;
        int64_t u = pw / R;
        int last_use[kMaxSlot];                    // last use this warp issued into each slot (drain)
        for (int i = 0; i < kMaxSlot; ++i) last_use[i] = -1;
        bool ok = true;
        for (int64_t j = pw; j < total_j; j += P) {
            if (u > 0 && !s_abort && !mbar_wait(&empty[slot], static_cast<uint32_t>((u - 1) & 1))) {
                set_error(a.err, kErrTimeout);
                s_abort = 1;
            }
            if (s_abort) { ok = false; break; }
            const int64_t tile = blockIdx.x + k * gridDim.x;
            const int s = tile_spectrum(a.tile_start, a.B, tile, a.tiles_per_spec, a.inv_tiles_per_spec);
            const int64_t nf = __ldg(a.nf_main + s);
            const int64_t n0 = (tile - __ldg(a.tile_start + s)) * Tn;
            const int64_t n_last = (n0 + Tn < nf ? n0 + Tn : nf) - 1;
            const int64_t base = __ldg(a.in_off + s);
            const int64_t avail = wp.extent - base;           // readable elements from x
            const T *x = static_cast<const T *>(a.x) + base;
            const int64_t g0 = static_cast<int64_t>(h) * n0;  // 16-byte aligned (n0 % 32 == 0)
            const int64_t g1 = static_cast<int64_t>(h) * n_last + h + 1;   // exclusive
            const int64_t g1u = (g1 + A - 1) & ~static_cast<int64_t>(A - 1);
            const int64_t gc = g1u <= avail ? g1u : (g1 & ~static_cast<int64_t>(A - 1));
            T *dst = reinterpret_cast<T *>(win_smem + static_cast<size_t>(slot) * wp.slot_bytes);
            uint32_t bytes = 0;
            if (gc > g0) {
                bytes = static_cast<uint32_t>((gc - g0) * static_cast<int64_t>(sizeof(T)));
                bulk_g2s(dst, x + g0, bytes, &full[slot]);
            }
            for (int64_t i = (gc > g0 ? gc : g0); i < g1; ++i) dst[i - g0] = x[i];   // unaligned tail
            mbar_arrive_expect_tx(&full[slot], bytes);
            last_use[slot] = static_cast<int>(u & 1) | 2;   // parity of the use, bit 1 = valid
            // advance to j + P
            h += P;
            while (h > H) { h -= H; ++k; }
            slot += P;
            if (slot >= R) { slot -= R; ++u; }
        }
        if (!ok) {
            // drain: wait (bounded) until the copies this warp issued have landed
            for (int i = 0; i < R; ++i)
                if (last_use[i] >= 0) mbar_wait(&full[i], static_cast<uint32_t>(last_use[i] & 1));
        }
        return;
    }

    // ------------------------------------------------------------------ consumers
    const int t = threadIdx.x;
    int cslot = 0;                    // slot of the next order (j % R) and its phase parity
    uint32_t cpar = 0;
    int loaded_spec = -1;
    for (int64_t k = 0; k < my_tiles; ++k) {
        const int64_t tile = blockIdx.x + k * gridDim.x;
        const int s = tile_spectrum(a.tile_start, a.B, tile, a.tiles_per_spec, a.inv_tiles_per_spec);
        if (s != loaded_spec) {
            consumer_sync(Tn);
            const int64_t no = a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0;
            for (int h = t; h < H; h += Tn) {
                if (kS) {
                    const float rs = __frcp_rn(__ldg(a.s.sigma + no + h));
                    nrm[0][h] = make_float2(rs, __fmul_rn(__ldg(a.s.mu + no + h), rs));
                }
                if (kG) {
                    const float rs = __frcp_rn(__ldg(a.g.sigma + no + h));
                    nrm[1][h] = make_float2(rs, __fmul_rn(__ldg(a.g.mu + no + h), rs));
                }
            }
            consumer_sync(Tn);
            loaded_spec = s;
        }
        const int64_t fbase = __ldg(a.fund_off + s);
        const int64_t nf = __ldg(a.nf_main + s);
        const int64_t n = (tile - __ldg(a.tile_start + s)) * Tn + t;
        const bool valid = n < nf;
        float best_s = 0.f, best_g = 0.f;
        int bh_s = 1, bh_g = 1;
        float ss = 0.f, sg = 0.f;
        int d = 0;
        uint32_t bits = 0;
        // order 1
        if (!s_abort && !mbar_wait(&full[cslot], cpar)) {
            set_error(a.err, kErrTimeout);
            s_abort = 1;
        }
        {
            const T *w = reinterpret_cast<const T *>(win_smem + static_cast<size_t>(cslot) * wp.slot_bytes);
            if (valid) {
                const float x0 = sm_ld<T>(w, t);
                ss = x0;
                sg = x0;
                if (kG && a.mitigation) {
                    const float x1 = sm_ld<T>(w, t + 1);
                    if (x1 > x0) { d = 1; sg = x1; bits = 1u; }
                }
                if (kS) { const float2 c = nrm[0][0]; best_s = fmaf(ss, c.x, -c.y); }
                if (kG) { const float2 c = nrm[1][0]; best_g = fmaf(sg, c.x, -c.y); }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[cslot]);
            if (++cslot == R) { cslot = 0; cpar ^= 1u; }
        }
        int e = t;                    // h t: element of this fundamental's h n in the window
        for (int h = 2; h <= H; ++h) {
            e += t;
            if (!s_abort && !mbar_wait(&full[cslot], cpar)) {
                set_error(a.err, kErrTimeout);
                s_abort = 1;
            }
            const T *w = reinterpret_cast<const T *>(win_smem + static_cast<size_t>(cslot) * wp.slot_bytes);
            if (valid) {
                if (kS) {
                    ss += sm_ld<T>(w, e);
                    const float2 c = nrm[0][h - 1];
                    const float v = fmaf(ss, c.x, -c.y);
                    if (v > best_s) { best_s = v; bh_s = h; }
                }
                if (kG) {
                    const float va = sm_ld<T>(w, e + d);
                    const float vb = sm_ld<T>(w, e + d + 1);
                    const bool inc = vb > va;
                    sg += inc ? vb : va;
                    d += inc;
                    bits |= static_cast<uint32_t>(inc) << (h - 1);
                    const float2 c = nrm[1][h - 1];
                    const float v = fmaf(sg, c.x, -c.y);
                    if (v > best_g) { best_g = v; bh_g = h; }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[cslot]);
            if (++cslot == R) { cslot = 0; cpar ^= 1u; }
        }
        if (valid && !s_abort) {
            const int64_t o = fbase + n;
            if (kS) {
                a.s.snr[o] = best_s;
                a.s.best_h[o] = static_cast<uint8_t>(bh_s);
            }
            if (kG) {
                a.g.snr[o] = best_g;
                a.g.best_h[o] = static_cast<uint8_t>(bh_g);
                if (a.g.path) store_path(a.g.path, a.path_bytes, o, bits);
            }
        }
        if (kS && a.s.argmax) consumer_argmax(valid ? argmax_key(best_s, n) : 0ull, a.s.argmax + s, red, Tn);
        if (kG && a.g.argmax) consumer_argmax(valid ? argmax_key(best_g, n) : 0ull, a.g.argmax + s, red, Tn);
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
