// Column-sweep 2D greedy sum (kernel 2 of a 2D plan); the schedule is described in
// hs_fwd2d_sweep.cuh, the per-order rule (shared with kernels 0 and 1) in hs_fwd2d.cuh.  Each
// chain takes the same steps in the same order as in the register-resident kernel, so the
// outputs are bit for bit those of kernels 0 and 1.
#include "hs_fwd1d.cuh"
#include "hs_fwd1d_win.cuh"
#include "hs_fwd2d.cuh"
#include "hs_fwd2d_sweep.cuh"

namespace hs {
namespace {

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Chain state between orders lives in L2 (L1 bypassed: other CTAs write it), kept there ahead of
// the streaming plane tiles by the `pol` eviction hint.
__device__ __forceinline__ int4 ld_state(const int4 *p, uint64_t pol)
{
    int4 v;
    asm volatile("ld.global.cg.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ void st_state(int4 *p, int4 v, uint64_t pol)
{
    asm volatile("st.global.cg.L2::cache_hint.v4.s32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}

// 2D tensor copy of the box at (x, y) into shared memory, completing on `bar` (expect-tx).
__device__ __forceinline__ void tensor_g2s_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                              uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// state word w: best order | (df + 8) << 8 | (dz + 8) << 16   (|df|, |dz| <= H - 1 <= 7)
__device__ __forceinline__ int4 pack_state(const Chain2D &c)
{
    return make_int4(__float_as_int(c.sum), __float_as_int(c.best), static_cast<int>(c.bits),
                     c.bh | ((c.df + 8) << 8) | ((c.dz + 8) << 16));
}

__device__ __forceinline__ Chain2D unpack_state(int4 v)
{
    Chain2D c;
    c.sum = __int_as_float(v.x);
    c.best = __int_as_float(v.y);
    c.bits = static_cast<uint32_t>(v.z);
    c.bh = v.w & 0xff;
    c.df = ((v.w >> 8) & 0xff) - 8;
    c.dz = ((v.w >> 16) & 0xff) - 8;
    return c;
}

// Bounded wait for phase `parity` of `bar`; false after kWaitNs or once another role has
// reported a failure (`dead`).
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, volatile int *dead)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (*dead) return false;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

// Push finished band jb (-1: no more) on the publisher's ring, waiting (bounded) while it is full.
__device__ __forceinline__ void push_finished(int *ring, volatile unsigned &head, volatile unsigned &tail, int jb,
                                              volatile int *dead, int *err)
{
    const unsigned h = head;
    if (h - tail >= static_cast<unsigned>(kSweepRing)) {
        const unsigned long long t0 = global_ns();
        while (h - tail >= static_cast<unsigned>(kSweepRing)) {
            if (*dead) return;
            if (global_ns() - t0 > kWaitNs) { set_error(err, kErrTimeout); *dead = 1; return; }
            __nanosleep(32);
        }
    }
    ring[h % kSweepRing] = jb;
    __threadfence_block();
    head = h + 1;
}

// Per-buffer description of the task staged in it (written by the control warp before it
// completes the buffer's `full` phase).
struct BandHdr {
    long long task;            // ticket; >= total: no more tasks
    long long c0;              // first anchor column of the band
    long long fa[kMaxH2D];     // order h = k + 1 holds chains [fa[k], fa[k] + nf[k]), all z
    int nf[kMaxH2D];
    int ev[kMaxH2D + 1];       // events of orders < h: order h's events are [ev[h-1], ev[h])
    unsigned mg[kMaxH2D];      // floor(2^32 / nf) + 1 for nf > 1 (0 for nf = 1): i / nf = (i mg) >> 32 for
                               // the event index i of an order (i nf < 2^32)
};
}  // namespace

template <typename T>
__global__ void __launch_bounds__(kSweepMaxThreads, 1) k_fwd2d_sweep(const __grid_constant__ CUtensorMap tmap,
                                                                   const Sweep2DArgs s)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ float rs[kMaxH2D], murs[kMaxH2D];
    __shared__ unsigned long long red[32];
    // full[b]: buffer b's plane tile has landed and the bands its chains' earlier orders lie in
    // are done (two arrivals of the control warp: the copy's, and one after the dependencies)
    __shared__ __align__(8) uint64_t full[kSweepMaxStages], empty[kSweepMaxStages];
    __shared__ BandHdr hdr[kSweepMaxStages];
    __shared__ int s_ring[kSweepRing];                  // finished bands, compute -> publisher
    __shared__ volatile unsigned s_head, s_tail;        // ring entries pushed / published
    __shared__ volatile int s_dead;
    __shared__ unsigned s_cnt[kSweepMaxStages];         // compute warps done with buffer b's task

    const Fwd2DArgs &a = s.a;
    const int H = a.H, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nz = static_cast<int>(a.nz);
    const int NC = blockDim.x - 64;                 // compute threads (warps 2..)
    const long long total = s.n_prefix + s.nbands;
    const int64_t f_hi = a.f_lo + a.nff - 1;
    unsigned *ticket = s.sync, *done = s.sync + 2;  // done[j]: band j
    if (tid < H) {
        const float r = __frcp_rn(__ldg(a.g.sigma + tid));
        rs[tid] = r;
        murs[tid] = __fmul_rn(__ldg(a.g.mu + tid), r);
    }
    const int nbuf = s.nbuf;
    if (tid == 0) {
        for (int i = 0; i < nbuf; ++i) {
            mbar_init(&full[i], 2);
            mbar_init(&empty[i], 1);
        }
        s_head = 0u;
        s_tail = 0u;
        s_dead = 0;
        for (int i = 0; i < kSweepMaxStages; ++i) s_cnt[i] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned long long key = 0ull;   // best argmax key of this thread's finished chains

    if (warp == 0) {
        // ---- control warp: task k goes to buffer b = k % nbuf (free once the compute warps
        // finished task k - nbuf).  It starts the copy of the band's plane tile into the buffer,
        // then waits until the bands holding the previous orders of the band's chains are done
        // (the compute warps read those chains' state from global memory).  Tickets are claimed
        // one task ahead, and the next band's table is built and its dependency flags are read
        // while the current band's copy is in flight.
        const uint64_t pol_plane = l2_policy_evict_first();
        const unsigned Wb = static_cast<unsigned>(s.Wb), band_lo = static_cast<unsigned>(s.band_lo);
        const unsigned f_s = static_cast<unsigned>(s.f_s), f_end = static_cast<unsigned>(f_hi + 1);
        unsigned pend = 0;                   // lane 0: buffers with copies not known to have landed
        uint32_t last_use[kSweepMaxStages] = {0u, 0u, 0u, 0u};
        auto claim = [&]() -> long long {
            return lane == 0 ? (s_dead ? total : static_cast<long long>(atomicAdd(ticket, 1u))) : 0ll;
        };
        // the prepared band: lane h - 1 holds order h; lane 2 (h - 2) + i (i = 0, 1) the i-th band
        // holding order h - 1 of order h's chains (p_dep = -1: none) with its flag as read
        long long pt = 0;
        unsigned p_fa = 0, p_nf = 0, p_flag = 1u;
        int p_c0 = 0, p_dep = -1;
        auto prepare = [&](long long t) {
            pt = t;
            p_nf = 0;
            p_fa = 0;
            p_dep = -1;
            p_flag = 1u;
            if (t < s.n_prefix || t >= total) return;
            const unsigned j = static_cast<unsigned>(t - s.n_prefix);
            const unsigned c0 = (band_lo + j) * Wb, c1 = c0 + Wb;
            int dlo = 0, dhi = -1;
            if (lane < H) {
                const unsigned h = lane + 1;
                unsigned fa = (c0 + h - 1) / h, fb = (c1 + h - 1) / h;
                fa = fa > f_s ? fa : f_s;
                fb = fb < f_end ? fb : f_end;
                p_nf = fb > fa ? fb - fa : 0u;
                p_fa = fa;
                if (h > 1 && p_nf > 0) {
                    dlo = static_cast<int>((h - 1) * fa / Wb - band_lo);
                    dhi = static_cast<int>((h - 1) * (fb - 1) / Wb - band_lo);
                }
            }
            p_c0 = static_cast<int>(c0);
            const int src = (lane >> 1) + 1 < kMaxH2D ? (lane >> 1) + 1 : 0;   // order h = src + 1 >= 2
            const int lo = __shfl_sync(0xffffffffu, dlo, src), hi = __shfl_sync(0xffffffffu, dhi, src);
            const int dep = lo + (lane & 1);
            if (lane < 2 * (kMaxH2D - 1) && dep <= hi) {
                if (dep < 0 || dep >= static_cast<int>(j)) set_error(a.err, kErrBounds);   // cannot happen, f_s >= Wb
                else {
                    p_dep = dep;
                    p_flag = ld_acquire(done + dep);
                }
            }
        };
        {
            long long t0 = claim();
            t0 = __shfl_sync(0xffffffffu, t0, 0);
            prepare(t0);
        }
        long long t_next = claim();
        for (long long k = 0;; ++k) {
            const int b = static_cast<int>(k % nbuf);
            const uint32_t u = static_cast<uint32_t>(k / nbuf);
            if (k >= nbuf) {
                int ok = 1;
                if (lane == 0) ok = wait_phase(&empty[b], (u - 1) & 1u, &s_dead) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) { set_error(a.err, kErrTimeout); s_dead = 1; }
                    break;
                }
                if (lane == 0) pend &= ~(1u << b);   // the compute warps waited on those copies
            }
            // one lane reads the failure flag, so the whole warp takes the same branch
            const int dead = __shfl_sync(0xffffffffu, lane == 0 ? static_cast<int>(s_dead) : 0, 0);
            const long long t = dead ? total : pt;
            if (t >= total || t < s.n_prefix) {
                if (lane == 0) {
                    hdr[b].task = t;
                    mbar_arrive(&full[b]);
                    mbar_arrive(&full[b]);
                }
                if (t >= total) break;
            } else {
                const int cnt = static_cast<int>(p_nf) * nz;
                // inclusive prefix over the orders of their event counts
                int einc = lane < H ? cnt : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int w = __shfl_up_sync(0xffffffffu, einc, o);
                    if (lane >= o) einc += w;
                }
                if (lane < H) {
                    hdr[b].fa[lane] = p_fa;
                    hdr[b].nf[lane] = static_cast<int>(p_nf);
                    hdr[b].mg[lane] = p_nf > 1 ? static_cast<unsigned>(0x100000000ull / p_nf + 1ull) : 0u;
                    hdr[b].ev[lane + 1] = einc;
                }
                if (lane == 0) {
                    hdr[b].task = t;
                    hdr[b].c0 = p_c0;
                    hdr[b].ev[0] = 0;
                }
                // the plane tile does not depend on other bands: its copy starts at once and the
                // dependency wait below overlaps it
                unsigned char *buf = dyn + static_cast<size_t>(b) * s.buf_bytes;
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[b], static_cast<uint32_t>(s.box_bytes));
                    tensor_g2s_2d(buf, &tmap, p_c0 - kSweepHalo, s.r_lo, &full[b], pol_plane);
                    pend |= 1u << b;
                    last_use[b] = u;
                }
                // dependencies: poll (bounded) the flags that were still clear when prepared
                bool unmet = false;
                if (p_dep >= 0 && p_flag == 0u) {
                    const unsigned long long t0 = global_ns();
                    while (ld_acquire(done + p_dep) == 0u) {
                        if (*reinterpret_cast<volatile int *>(a.err) == kErrTimeout) { unmet = true; break; }
                        if (global_ns() - t0 > kWaitNs) { set_error(a.err, kErrTimeout); unmet = true; break; }
                        __nanosleep(64);
                    }
                }
                // a band whose dependencies were not met would read chain state that was never
                // written (its drift could point outside the staged tile): the CTA stops instead,
                // handing the compute warps the end marker
                const bool stop = __any_sync(0xffffffffu, unmet);
                if (stop && lane == 0) {
                    s_dead = 1;
                    hdr[b].task = total;
                }
                // the second arrival follows every lane's acquire of its flag (warp barrier), so
                // the compute warps, which wait for it, see the state those bands stored
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[b]);
                __syncwarp();
                if (stop) break;
            }
            // the next task: its ticket was claimed one task ago
            long long tn = __shfl_sync(0xffffffffu, t_next, 0);
            if (tn < total) t_next = claim();
            prepare(tn);
        }
        // copies of a buffer the compute warps never waited on (after a failure) land first
        if (lane == 0)
            for (int i = 0; i < nbuf; ++i)
                if (pend & (1u << i)) {
                    volatile int never = 0;
                    wait_phase(&full[i], last_use[i] & 1u, &never);
                }
        __syncwarp();
    } else if (warp == 1) {
        // ---- publisher: mark finished bands done.  The last compute warp done with a band pushes
        // it on a shared ring; one GPU-scope fence then covers every band pushed so far (every
        // warp's state stores were ordered before the push by the block-scope release / acquire
        // of the warps' done count), so a fence per batch rather than per band sets the flags.
        if (lane == 0) {
            unsigned tail = 0u;
            bool end = false;
            while (!end) {
                unsigned head = s_head;
                if (head == tail) {
                    const unsigned long long t0 = global_ns();
                    while ((head = s_head) == tail) {
                        if (s_dead) break;
                        if (global_ns() - t0 > kWaitNs) { set_error(a.err, kErrTimeout); s_dead = 1; break; }
                        __nanosleep(32);
                    }
                    if (head == tail) break;
                }
                __threadfence();
                for (; tail != head; ++tail) {
                    const int jb = s_ring[tail % kSweepRing];
                    if (jb < 0) { end = true; break; }
                    st_release(done + jb, 1u);
                }
                s_tail = tail;
            }
        }
        __syncwarp();
    } else {
        // ---- compute warps: run task k from buffer k % nbuf.  Each warp goes through the tasks on
        // its own (no barrier across the compute warps): the last warp to finish a task releases
        // its buffer to the control warp and hands the band to the publisher.
        const int ctid = tid - 64;
        const unsigned NW = static_cast<unsigned>(NC >> 5);
        // state kept in L2 ahead of the tiles (evict-last), except the last read of a chain's state
        // (order H reads order H - 1's): evict-first, so no dead state outlives the pass in L2
        const uint64_t pol_state = l2_policy_evict_last(), pol_dead = l2_policy_evict_first();
        const int P = s.Wb + 2 * kSweepHalo;
        int rot = 0;   // events of the bands so far, mod NC (the bands' events form one round-robin)
        for (long long k = 0;; ++k) {
            const int b = static_cast<int>(k % nbuf);
            const uint32_t u = static_cast<uint32_t>(k / nbuf);
            const bool lost = !wait_phase(&full[b], u & 1u, &s_dead);
            if (__any_sync(0xffffffffu, lost)) {
                if (lane == 0) { set_error(a.err, kErrTimeout); s_dead = 1; }
                break;
            }
            const BandHdr &hd = hdr[b];
            const long long t = hd.task;
            int jb = -2;   // what the last warp hands to the publisher: band j, -1 (end) or nothing
            if (t >= total) {
                jb = -1;
            } else if (t < s.n_prefix) {
                // prefix task: chains f < f_s, each carried in registers through all orders
                const long long npf = s.f_s - a.f_lo;
                const long long c = t * NC + ctid;
                if (c < npf * nz) {
                    const long long zi = c / npf, fi = c % npf;
                    const long long f = a.f_lo + fi, z = a.z_lo + zi;
                    Chain2D ch{0.f, 0.f, 0u, 0, 0, 1};
                    for (int h = 1; h <= H; ++h) {
                        const long long cf = h * f + ch.df, cr = a.z0_row + h * z + ch.dz;
                        const T *r0 = static_cast<const T *>(a.plane) + (cr - 1) * a.n_freq + cf;
                        float v9[9];
#pragma unroll
                        for (int r = 0; r < 3; ++r)
#pragma unroll
                            for (int q = 0; q < 3; ++q) v9[3 * r + q] = ld_raw<T, int64_t>(r0 + r * a.n_freq, q - 1);
                        chain2d_step(ch, h, v9, rs[h - 1], murs[h - 1]);
                    }
                    const long long o = zi * a.nff + fi;
                    a.g.snr[o] = ch.best;
                    a.g.best_h[o] = static_cast<uint8_t>(ch.bh);
                    if (a.g.path) static_cast<uint32_t *>(a.g.path)[o] = ch.bits;
                    const unsigned long long kk = argmax_key(ch.best, o);
                    key = kk > key ? kk : key;
                }
            } else {
                jb = static_cast<int>(t - s.n_prefix);
                const unsigned char *buf = dyn + static_cast<size_t>(b) * s.buf_bytes;
                const T *tile = reinterpret_cast<const T *>(buf);
                const int col0 = static_cast<int>(hd.c0 - kSweepHalo);   // plane column of tile column 0
                // the band's events of every order as one index space e in [0, ev[H]): order h holds
                // [ev[h-1], ev[h]), within it event i is chain (fa + i % nf, z_lo + i / nf).  Every
                // event of a band is independent of the others (order h of chain f anchors at h f,
                // order h + 1 at h f + f >= h f + Wb: a later band), so the orders need no barrier
                // between them.  The events of successive bands continue one round-robin over the
                // compute threads, so no thread idles at the end of a band.  A thread's events
                // increase, so its order h only moves up.  The states of a thread's next two events
                // are loaded (from L2) while it computes the current one.
                const int E = hd.ev[H];
                int e = ctid - rot;
                if (e < 0) e += NC;
                rot = (rot + E) % NC;
                int h = 0, e_lo = 0, e_hi = 0, nf = 0, fa = 0;
                unsigned mg = 0u;
                // event ee -> order hh, chain fh, row index zh (z - z_lo)
                auto decode = [&](int ee, int &hh, int &fh, int &zh) {
                    if (ee >= e_hi) {
                        do {
                            ++h;
                            e_lo = e_hi;
                            e_hi = hd.ev[h];
                        } while (ee >= e_hi);
                        nf = hd.nf[h - 1];
                        fa = static_cast<int>(hd.fa[h - 1]);
                        mg = hd.mg[h - 1];
                    }
                    const unsigned i = static_cast<unsigned>(ee - e_lo);
                    zh = nf > 1 ? static_cast<int>(__umulhi(i, mg)) : static_cast<int>(i);
                    fh = fa + (static_cast<int>(i) - zh * nf);
                    hh = h;
                };
                // state entry of chain (fh, z_lo + zh): fewer than 2^31 entries (the host checks)
                const unsigned nfs32 = static_cast<unsigned>(s.nfs), fs32 = static_cast<unsigned>(s.f_s);
                auto state_at = [&](int fh, int zh) {
                    return s.state + (static_cast<unsigned>(zh) * nfs32 + (static_cast<unsigned>(fh) - fs32));
                };
                if (e < E) {
                    int hc, fc, zc, hn = 0, fn = 0, zn = 0;
                    decode(e, hc, fc, zc);
                    int4 sc = hc > 1 ? ld_state(state_at(fc, zc), hc == H ? pol_dead : pol_state) : make_int4(0, 0, 0, 0);
                    int4 sn = make_int4(0, 0, 0, 0);
                    if (e + NC < E) {
                        decode(e + NC, hn, fn, zn);
                        if (hn > 1) sn = ld_state(state_at(fn, zn), hn == H ? pol_dead : pol_state);
                    }
                    for (;;) {
                        const int e2 = e + 2 * NC;
                        int h2 = 0, f2 = 0, z2 = 0;
                        int4 s2 = make_int4(0, 0, 0, 0);
                        if (e2 < E) {
                            decode(e2, h2, f2, z2);
                            if (h2 > 1) s2 = ld_state(state_at(f2, z2), h2 == H ? pol_dead : pol_state);
                        }
                        Chain2D ch{0.f, 0.f, 0u, 0, 0, 1};
                        if (hc > 1) ch = unpack_state(sc);
                        const int zrow = static_cast<int>(a.z0_row) + hc * static_cast<int>(a.z_lo) - 1 - s.r_lo;
                        const int cf = hc * fc + ch.df;
                        const int cr = zrow + hc * zc + ch.dz;   // staged row of the neighbourhood's top row
                        const T *p0 = tile + cr * P + (cf - 1 - col0);
                        float v9[9];
#pragma unroll
                        for (int r = 0; r < 3; ++r)
#pragma unroll
                            for (int q = 0; q < 3; ++q) v9[3 * r + q] = sm_ld<T>(p0 + r * P, q);
                        chain2d_step(ch, hc, v9, rs[hc - 1], murs[hc - 1]);
                        if (hc == H) {
                            const long long o = static_cast<long long>(zc) * a.nff + (fc - a.f_lo);
                            a.g.snr[o] = ch.best;
                            a.g.best_h[o] = static_cast<uint8_t>(ch.bh);
                            if (a.g.path) static_cast<uint32_t *>(a.g.path)[o] = ch.bits;
                            const unsigned long long kx = argmax_key(ch.best, o);
                            key = kx > key ? kx : key;
                        } else {
                            st_state(state_at(fc, zc), pack_state(ch), pol_state);
                        }
                        if (e + NC >= E) break;
                        e += NC;
                        hc = hn;
                        fc = fn;
                        zc = zn;
                        sc = sn;
                        hn = h2;
                        fn = f2;
                        zn = z2;
                        sn = s2;
                    }
                }
            }
            // this warp is done with the buffer and its stores are issued; the last warp of the
            // task (its count, taken with release / acquire fences at block scope, orders every
            // warp's stores before it) releases the buffer and hands the band to the publisher
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                const unsigned c = atomicAdd(&s_cnt[b], 1u);
                if (c + 1u == NW) {
                    __threadfence_block();
                    s_cnt[b] = 0u;
                    if (jb != -2) push_finished(s_ring, s_head, s_tail, jb, &s_dead, a.err);
                    if (jb != -1) mbar_arrive(&empty[b]);
                }
            }
            __syncwarp();
            if (t >= total) break;
        }
    }
    __syncthreads();
    if (a.g.argmax) block_argmax(key, a.g.argmax, red);
}

const void *fwd2d_sweep_kernel(int dtype)
{
    switch (dtype) {
    case HS_F32: return reinterpret_cast<const void *>(&k_fwd2d_sweep<float>);
    case HS_F16: return reinterpret_cast<const void *>(&k_fwd2d_sweep<__half>);
    case HS_BF16: return reinterpret_cast<const void *>(&k_fwd2d_sweep<__nv_bfloat16>);
    }
    return nullptr;
}

}  // namespace hs
