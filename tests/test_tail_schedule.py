"""CPU checks of the tiling the truncated tail (HS_FLAG_TRUNCATE_TAIL) relies on, derived from the
tail rule itself: fundamental n of a spectrum of N bins keeps the simple orders h with h n <= N - 1
and the greedy orders with h n + h <= N - 1.  The tail N_f <= n < N - 1 (N_f = floor((N - 1) / H))
is split at n1 = floor((N - 1) / 2) + 1 into generic tiles of 1024 fundamentals (N_f <= n < n1) and
one-order tiles of 8192 (n1 <= n < N - 1); spectrum s owns G_s + O_s consecutive CTAs of one launch
(its generic tiles, then its one-order tiles), and a CTA finds its spectrum by a division when all
spectra share one length, else by a binary search over the summed tile prefixes.  Checked for
several batch shapes: the CTA numbering is inverted exactly, every tail fundamental lies in exactly
one tile, both forms keep exactly one order in every one-order tile, and every read stays below N."""
import numpy as np
import pytest

GENERIC_TILE = 1024
ONE_ORDER_TILE = 8192


def ceil_div(a, b):
    return -(-a // b)


def tables(lengths, H):
    """Generic and one-order tile prefixes of a batch (the plan's host tables)."""
    g = [0]
    o = [0]
    for N in lengths:
        nf_main, nf, n1 = (N - 1) // H, N - 1, (N - 1) // 2 + 1
        g.append(g[-1] + ceil_div(max(0, min(nf, n1) - nf_main), GENERIC_TILE))
        o.append(o[-1] + ceil_div(max(0, nf - max(n1, nf_main)), ONE_ORDER_TILE))
    return np.array(g, np.int64), np.array(o, np.int64)


def cta_spectrum(q, g, o, equal):
    """Spectrum and first combined index of the CTAs that hold combined index q."""
    B = len(g) - 1
    if B == 1:
        return 0, 0
    if equal:
        per = int(g[-1] // B + o[-1] // B)
        s = min(q // per, B - 1)
        return s, s * per
    lo, hi = 0, B - 1
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if g[mid] + o[mid] <= q:
            lo = mid
        else:
            hi = mid - 1
    return lo, int(g[lo] + o[lo])


@pytest.mark.parametrize("lengths,H", [([131072] * 12, 32), ([131072] * 3, 2), ([4097, 70001, 33, 2050, 34], 32),
                                       ([5000, 40000, 20011, 9000], 16), ([3] * 5, 2), ([5, 4, 3], 2),
                                       ([1 << 20], 32), ([1 << 20] * 2, 8), ([20000], 1), ([9, 17, 100000, 12], 7)])
def test_tail_tiling(lengths, H):
    g, o = tables(lengths, H)
    equal = len(set(lengths)) == 1
    total = int(g[-1] + o[-1])
    seen = [np.zeros(N, np.int32) for N in lengths]
    for block in range(total):
        q = total - 1 - block                      # the launch runs the last spectrum first
        s, c0 = cta_spectrum(q, g, o, equal)
        assert int(g[s] + o[s]) <= q < int(g[s + 1] + o[s + 1])
        assert c0 == int(g[s] + o[s])
        N = lengths[s]
        nf_main, nf, n1 = (N - 1) // H, N - 1, (N - 1) // 2 + 1
        j, gn = q - c0, int(g[s + 1] - g[s])
        if j < gn:
            lo = nf_main + j * GENERIC_TILE
            ns = np.arange(lo, min(lo + GENERIC_TILE, min(nf, n1)))
            assert ns.size > 0
            # simple reads h n <= N - 1, greedy h n + d, h n + d + 1 <= h n + h <= N - 1
            hs = np.minimum((N - 1) // ns, H)
            hg = np.minimum((N - 1) // (ns + 1), H)
            assert np.all(hs * ns <= N - 1) and np.all(hg * ns + hg <= N - 1)
        else:
            lo = max(n1, nf_main) + (j - gn) * ONE_ORDER_TILE
            ns = np.arange(lo, min(lo + ONE_ORDER_TILE, nf))
            assert ns.size > 0
            # both forms keep order 1 only; order 1 reads x[n] and x[n + 1]
            assert np.all((N - 1) // ns == 1) and np.all((N - 1) // (ns + 1) == 1)
            assert np.all(ns + 1 <= N - 1)
        seen[s][ns] += 1
    for N, c in zip(lengths, seen):
        nf_main = (N - 1) // H
        assert np.all(c[:nf_main] == 0) and np.all(c[nf_main:N - 1] == 1) and c[N - 1] == 0


def test_generic_tile_chain_mapping():
    """Within a generic tile, warp w runs fundamentals [128 w, 128 w + 128) and lane l's chain c is
    32 c + l of them: the 256 threads x 4 chains cover the 1024 fundamentals of the tile once, and a
    thread's chains lie within 96 fundamentals of each other."""
    threads, chains = 256, 4
    assert threads * chains == GENERIC_TILE
    seen = np.zeros(GENERIC_TILE, np.int32)
    for t in range(threads):
        ns = [(t >> 5) * (32 * chains) + c * 32 + (t & 31) for c in range(chains)]
        assert max(ns) - min(ns) == 32 * (chains - 1)
        for n in ns:
            seen[n] += 1
    assert np.all(seen == 1)
