"""CPU checks of the schedule the 2D column sweep (kernel 2) relies on, derived from the 2D rule
itself: order h of chain (f, z) is centred at (h f + df, h z + dz) with |df|, |dz| <= h - 1 and reads
its 3x3 neighbourhood.  Band j of width Wb holds the events whose anchor h f lies in
[j Wb, j Wb + Wb); the sweep starts at f_s = 64 Wb and stages the band's columns widened by 8 on
each side and every row a chain can reach.  Checked for several plane shapes: every (f, h) of the
sweep lies in exactly one band, a chain's orders lie in strictly increasing bands, the previous
order of a band's order-h chains lies in at most two bands, all before it, every read of a band's
events falls inside its staged tile, and the plan's workspace is 16 bytes per swept chain plus one
flag per band (rounded to 256 bytes) for the narrowest band, 16 columns."""
import numpy as np
import pytest

HALO = 8


@pytest.fixture(scope="module")
def hs():
    """The binding (built in-tree first), for host-only plans (HS_FLAG_NO_DEVICE): no GPU needed."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_2202_12817_gb300 as hs_mod
    return hs_mod


def ceil_div(a, b):
    return -(-a // b)


def staged_rows(z0, H, z_lo, z_hi, n_rows):
    lo = min(z0 + h * z_lo - h for h in range(1, H + 1))
    hi = max(z0 + h * z_hi + h for h in range(1, H + 1))
    return max(lo, 0), min(hi, n_rows - 1)


@pytest.mark.parametrize("n_freq,n_rows,z0,H,Wb", [(1 << 17, 201, 100, 8, 64), (1 << 17, 201, 100, 8, 96),
                                                   (1 << 17, 201, 100, 8, 112), (1 << 17, 201, 100, 8, 128),
                                                   (40000, 61, 30, 4, 16), (65536, 23, 11, 3, 32),
                                                   (2404, 9, 4, 2, 16), (33000, 201, 150, 6, 64),
                                                   (100000, 9, 4, 1, 64)])
def test_band_schedule(hs, n_freq, n_rows, z0, H, Wb):
    plan = hs.Plan(H, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=n_rows, z0_row=z0, flags=hs.FLAG_NO_DEVICE)
    f_lo, f_hi, z_lo, z_hi = plan.domain
    plan.close()
    f_s = max(f_lo, 64 * Wb)
    assert f_s <= f_hi
    band_lo = f_s // Wb
    nbands = H * f_hi // Wb - band_lo + 1
    r_lo, r_hi = staged_rows(z0, H, z_lo, z_hi, n_rows)
    band_of = {}
    for j in range(nbands):
        c0 = (band_lo + j) * Wb
        c1 = c0 + Wb
        x0 = c0 - HALO                      # first staged column
        assert x0 >= 0
        for h in range(1, H + 1):
            fa, fb = max(ceil_div(c0, h), f_s), min(ceil_div(c1, h), f_hi + 1)
            if fb <= fa:
                continue
            f = np.arange(fa, fb)
            assert np.all((h * f >= c0) & (h * f < c1))
            # columns and rows any drift can reach stay inside the staged tile
            assert h * fa - h >= x0 and h * (fb - 1) + h < c1 + HALO
            assert z0 + h * z_lo - h >= r_lo and z0 + h * z_hi + h <= r_hi
            for ff in f.tolist():
                assert (ff, h) not in band_of
                band_of[(ff, h)] = j
            if h > 1:
                dlo = (h - 1) * fa // Wb - band_lo
                dhi = (h - 1) * (fb - 1) // Wb - band_lo
                assert 0 <= dlo <= dhi <= dlo + 1 and dhi < j
    assert len(band_of) == (f_hi - f_s + 1) * H
    for ff in range(f_s, f_hi + 1):
        bands = [band_of[(ff, h)] for h in range(1, H + 1)]
        assert all(bands[i] < bands[i + 1] for i in range(H - 1))


@pytest.mark.parametrize("n_freq,n_rows,z0,H,dtype", [(1 << 21, 201, 100, 8, 0), (1 << 21, 201, 100, 8, 1),
                                                      (80000, 61, 30, 8, 0), (65536, 49, 24, 3, 2)])
def test_workspace_size(hs, n_freq, n_rows, z0, H, dtype):
    plan = hs.Plan(H, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=n_rows, z0_row=z0, dtype=dtype,
                   flags=hs.FLAG_NO_DEVICE)
    f_lo, f_hi, z_lo, z_hi = plan.domain
    f_s = max(f_lo, 64 * 16)
    nbands = H * f_hi // 16 - f_s // 16 + 1
    expect = (z_hi - z_lo + 1) * (f_hi - f_s + 1) * 16 + ceil_div(4 * (2 + nbands), 256) * 256
    assert plan.workspace_bytes == expect
    plan.close()
