/*
 * hs_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 reference for the incoherent harmonic sum of
 * Adamek, Roy & Armour, "A Novel Greedy Approach To Harmonic Summing Using GPUs"
 * (arXiv:2202.12817).  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library.  It shares no code, header or constant with
 * the CUDA path.
 *
 * Conventions used throughout (the paper's notation, 0-based bins):
 *   x[j]   loaded power of bin j; p[j] promoted exactly to double, or with a per-bin
 *          whitening weight w[j] the product w[j]*p[j] rounded once to FP32 (round_w != 0)
 *          or kept exact in FP64 (round_w == 0, used by finite-difference checks);
 *   n      fundamental bin, n in [0, nf) with nf = floor((N-1)/H): the largest domain in
 *          which every read of both forms (greedy max index H*n + H) stays inside the
 *          spectrum -- the paper's "every frequency bin up to a limit" (Sec. 2);
 *   h      harmonic order 1..H, h = 1 being the fundamental;
 *   mu[h-1], sigma[h-1]   mean and standard deviation of a partial sum of h terms (Eq. 2).
 *
 * Returns 0 on success, -1 on invalid arguments.
 *
 * The loops over fundamentals of the 1D simple and greedy forms and of the 2D form carry an
 * OpenMP pragma.  The oracle proper (liboracle.so) is compiled without OpenMP, so the pragma is
 * ignored and everything runs on one thread; the CPU baseline of the benchmark also times a
 * second build with OpenMP (liboracle_omp.so), the same arithmetic spread over the host's cores
 * (every fundamental is independent and writes only its own outputs).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HSO_MAX_H 32

static double load_x(const float *p, const float *w, int32_t round_w, int64_t j)
{
    if (!w) return (double)p[j];
    double prod = (double)w[j] * (double)p[j]; /* exact: 24+24 significant bits */
    return round_w ? (double)(float)prod : prod;
}

int64_t hso_nf_1d(int64_t n, int32_t H)
{
    if (H < 1 || H > HSO_MAX_H || n < (int64_t)H + 1) return 0;
    return (n - 1) / H;
}

/* Eq. 2: SNR of a partial sum of h terms. */
static double snr_of(double sum, int h, const double *mu, const double *sigma)
{
    return (sum - mu[h - 1]) / sigma[h - 1];
}

/*
 * Simple harmonic sum, Eq. 3: X_h[n] = sum_{k=1..h} x[k n], followed by Eq. 2's maximum
 * over the partial sums h = 1..H.  The running maximum starts at h = 1 and is replaced
 * only by a strictly larger SNR, so the lowest h wins ties.
 */
int hso_simple_1d(const float *p, const float *w, int32_t round_w, int64_t n, int32_t H,
                  const double *mu, const double *sigma, int64_t nf,
                  double *snr, uint8_t *best_h, double *snr_all)
{
    if (!p || !mu || !sigma || H < 1 || H > HSO_MAX_H || nf < 0) return -1;
    if (nf > hso_nf_1d(n, H)) return -1;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t f = 0; f < nf; ++f) {
        double sum = 0.0, best = 0.0;
        int bh = 0;
        for (int h = 1; h <= H; ++h) {
            sum += load_x(p, w, round_w, (int64_t)h * f);
            double s = snr_of(sum, h, mu, sigma);
            if (snr_all) snr_all[f * H + (h - 1)] = s;
            if (h == 1 || s > best) { best = s; bh = h; }
        }
        if (snr) snr[f] = best;
        if (best_h) best_h[f] = (uint8_t)bh;
    }
    return 0;
}

/*
 * Greedy harmonic sum, Eq. 5 and Algorithm 2.
 *   Order 1 (the fundamental): with scalloping-loss mitigation the values of bins n and
 *   n+1 are compared; if bin n+1 is strictly larger the drift becomes 1 and its value is
 *   summed, else bin n is summed.  Without mitigation bin n is summed and d stays 0.
 *   Orders h = 2..H: m = h n + d; if x[m+1] > x[m] (strictly) then d <- d+1 and x[m+1] is
 *   summed, else x[m] is summed.
 * Bit h-1 of path[n] records an increment at order h, so the bin chosen at order k is
 * k n + popcount(path & ((1 << k) - 1)).
 */
static void greedy_one(const float *p, const float *w, int32_t round_w, int32_t H, int32_t mitigation,
                       const double *mu, const double *sigma, int64_t f, double *snr, uint8_t *best_h,
                       uint32_t *path, double *snr_all_row)
{
    int64_t d = 0;
    uint32_t bits = 0;
    double sum;
    if (mitigation) {
        double a = load_x(p, w, round_w, f), b = load_x(p, w, round_w, f + 1);
        if (b > a) { d = 1; sum = b; bits |= 1u; }
        else { sum = a; }
    } else {
        sum = load_x(p, w, round_w, f);
    }
    double best = snr_of(sum, 1, mu, sigma);
    int bh = 1;
    if (snr_all_row) snr_all_row[0] = best;
    for (int h = 2; h <= H; ++h) {
        int64_t m = (int64_t)h * f + d;
        double a = load_x(p, w, round_w, m), b = load_x(p, w, round_w, m + 1);
        if (b > a) { d += 1; sum += b; bits |= 1u << (h - 1); }
        else { sum += a; }
        double s = snr_of(sum, h, mu, sigma);
        if (snr_all_row) snr_all_row[h - 1] = s;
        if (s > best) { best = s; bh = h; }
    }
    if (snr) *snr = best;
    if (best_h) *best_h = (uint8_t)bh;
    if (path) *path = bits;
}

int hso_greedy_1d(const float *p, const float *w, int32_t round_w, int64_t n, int32_t H,
                  int32_t mitigation, const double *mu, const double *sigma, int64_t nf,
                  double *snr, uint8_t *best_h, uint32_t *path, double *snr_all)
{
    if (!p || !mu || !sigma || H < 1 || H > HSO_MAX_H || nf < 0) return -1;
    if (nf > hso_nf_1d(n, H)) return -1;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t f = 0; f < nf; ++f)
        greedy_one(p, w, round_w, H, mitigation, mu, sigma, f, snr ? snr + f : NULL, best_h ? best_h + f : NULL,
                   path ? path + f : NULL, snr_all ? snr_all + f * H : NULL);
    return 0;
}

/*
 * The greedy form above for the `count` fundamentals listed in fund[] (each in [0, nf)), outputs
 * in list order.  Used where only a few fundamentals can change, e.g. the fundamentals whose
 * reads may include one perturbed bin in a finite-difference check.
 */
int hso_greedy_1d_list(const float *p, const float *w, int32_t round_w, int64_t n, int32_t H,
                       int32_t mitigation, const double *mu, const double *sigma, int64_t count,
                       const int64_t *fund, double *snr, uint8_t *best_h, uint32_t *path)
{
    if (!p || !mu || !sigma || !fund || H < 1 || H > HSO_MAX_H || count < 0) return -1;
    const int64_t nf = hso_nf_1d(n, H);
    for (int64_t i = 0; i < count; ++i)
        if (fund[i] < 0 || fund[i] >= nf) return -1;
    for (int64_t i = 0; i < count; ++i)
        greedy_one(p, w, round_w, H, mitigation, mu, sigma, fund[i], snr ? snr + i : NULL,
                   best_h ? best_h + i : NULL, path ? path + i : NULL, NULL);
    return 0;
}

/*
 * Fundamentals past the full-harmonic domain: n in [lo, hi) with N_f <= lo and hi <= N - 1 (the
 * reading of "for each bin" that keeps every bin whose fundamental comparison fits, Sec. 1 and
 * Algorithm 2's loop over the spectrum).  Each form sums only the orders whose every possible
 * read lies inside the spectrum:
 *   simple (form 1): the bin of order h is h n, so H_n = min(H, floor((N-1)/n));
 *   greedy (form 2) and optimal (form 4): the bins of order h are at most h n + h (drift at most
 *   h - 1 after order h - 1, plus the compared neighbour), so H_n = min(H, floor((N-1)/(n+1))).
 * Within its H_n orders each form is exactly the one above (Eq. 3; Eq. 5 / Algorithm 2; the
 * optimum of hso_dp_1d), and the maximum of Eq. 2 runs over h = 1..H_n.  snr_all [hi-lo][H]
 * (may be NULL) holds NaN for the excluded orders; path (greedy only, may be NULL).
 */
int hso_dp_1d(const float *p, const float *w, int32_t round_w, int64_t n, int32_t H,
              int32_t mitigation, int64_t fund, double *best_sum);

static int64_t tail_orders(int32_t form, int64_t n, int32_t H, int64_t f)
{
    const int64_t lim = form == 1 ? (f == 0 ? H : (n - 1) / f) : (n - 1) / (f + 1);
    return lim < H ? lim : H;
}

int hso_tail_1d(int32_t form, const float *p, const float *w, int32_t round_w, int64_t n, int32_t H,
                int32_t mitigation, const double *mu, const double *sigma, int64_t lo, int64_t hi,
                double *snr, uint8_t *best_h, uint32_t *path, double *snr_all)
{
    if (!p || !mu || !sigma || H < 1 || H > HSO_MAX_H || lo < 0 || hi > n - 1 || lo > hi) return -1;
    if (form != 1 && form != 2 && form != 4) return -1;
    for (int64_t f = lo; f < hi; ++f) {
        const int64_t i = f - lo;
        const int Hn = (int)tail_orders(form, n, H, f);
        if (Hn < 1) return -1;
        double sums[HSO_MAX_H];
        uint32_t bits = 0;
        if (form == 1) {
            double sum = 0.0;
            for (int h = 1; h <= Hn; ++h) {
                sum += load_x(p, w, round_w, (int64_t)h * f);
                sums[h - 1] = sum;
            }
        } else if (form == 2) {
            int64_t d = 0;
            double sum;
            if (mitigation) {
                double a = load_x(p, w, round_w, f), b = load_x(p, w, round_w, f + 1);
                if (b > a) { d = 1; sum = b; bits |= 1u; }
                else { sum = a; }
            } else {
                sum = load_x(p, w, round_w, f);
            }
            sums[0] = sum;
            for (int h = 2; h <= Hn; ++h) {
                const int64_t m = (int64_t)h * f + d;
                double a = load_x(p, w, round_w, m), b = load_x(p, w, round_w, m + 1);
                if (b > a) { d += 1; sum += b; bits |= 1u << (h - 1); }
                else { sum += a; }
                sums[h - 1] = sum;
            }
        } else {
            if (hso_dp_1d(p, w, round_w, n, Hn, mitigation, f, sums) != 0) return -1;
        }
        double best = snr_of(sums[0], 1, mu, sigma);
        int bh = 1;
        for (int h = 1; h <= H; ++h) {
            const double v = h <= Hn ? snr_of(sums[h - 1], h, mu, sigma) : NAN;
            if (snr_all) snr_all[i * H + (h - 1)] = v;
            if (h > 1 && h <= Hn && v > best) { best = v; bh = h; }
        }
        if (snr) snr[i] = best;
        if (best_h) best_h[i] = (uint8_t)bh;
        if (path && form == 2) path[i] = bits;
    }
    return 0;
}

/*
 * 2D greedy harmonic sum over an f-fdot plane (the higher-dimensional harmonic sum the
 * paper names for acceleration searches; the paper gives no 2D algorithm, so this
 * follows the 1D rule lifted to a 3x3 neighbourhood):
 *   plane is row-major [n_rows][n_freq], row r = z0_row + z;
 *   (df, dz) = (0, 0); for h = 1..H the centre is (h f + df, h z + dz); the best value
 *   starts at the centre and the 8 neighbours are scanned in raster order (dz = -1, 0, 1
 *   outer; df = -1, 0, 1 inner), each replacing the best only if strictly larger; the
 *   best value is summed and (df, dz) moves by the winning offset.  The 4-bit code of
 *   order h, (oz + 1) * 3 + (of + 1), is stored at bits 4(h-1)..4h-1 of path (4 = centre).
 * Output index = (z - z_lo) * (f_hi - f_lo + 1) + (f - f_lo).
 */
int hso_greedy_2d(const float *plane, int64_t n_freq, int64_t n_rows, int64_t z0_row, int32_t H,
                  int64_t f_lo, int64_t f_hi, int64_t z_lo, int64_t z_hi,
                  const double *mu, const double *sigma,
                  double *snr, uint8_t *best_h, uint32_t *path, double *snr_all)
{
    if (!plane || !mu || !sigma || H < 1 || H > 8) return -1;
    if (f_lo < 1 || f_hi < f_lo || z_hi < z_lo) return -1;
    /* every read must lie inside the plane: check the extreme orders 1 and H */
    if ((int64_t)H * f_hi + H > n_freq - 1) return -1;
    for (int hh = 1; hh <= H; hh += (H > 1 ? H - 1 : 1)) {
        if (z0_row + (int64_t)hh * z_lo - hh < 0) return -1;
        if (z0_row + (int64_t)hh * z_hi + hh > n_rows - 1) return -1;
    }
    const int64_t nff = f_hi - f_lo + 1;
#pragma omp parallel for collapse(2) schedule(dynamic, 1024)
    for (int64_t z = z_lo; z <= z_hi; ++z) {
        for (int64_t f = f_lo; f <= f_hi; ++f) {
            const int64_t o = (z - z_lo) * nff + (f - f_lo);
            int64_t df = 0, dz = 0;
            double sum = 0.0, best = 0.0;
            uint32_t bits = 0;
            int bh = 0;
            for (int h = 1; h <= H; ++h) {
                const int64_t cf = (int64_t)h * f + df;
                const int64_t cr = z0_row + (int64_t)h * z + dz;
                double v = (double)plane[cr * n_freq + cf];
                int bf = 0, bz = 0;
                for (int oz = -1; oz <= 1; ++oz) {
                    for (int of = -1; of <= 1; ++of) {
                        if (oz == 0 && of == 0) continue;
                        double c = (double)plane[(cr + oz) * n_freq + (cf + of)];
                        if (c > v) { v = c; bf = of; bz = oz; }
                    }
                }
                sum += v;
                df += bf;
                dz += bz;
                bits |= (uint32_t)((bz + 1) * 3 + (bf + 1)) << (4 * (h - 1));
                double s = snr_of(sum, h, mu, sigma);
                if (snr_all) snr_all[o * H + (h - 1)] = s;
                if (h == 1 || s > best) { best = s; bh = h; }
            }
            if (snr) snr[o] = best;
            if (best_h) best_h[o] = (uint8_t)bh;
            if (path) path[o] = bits;
        }
    }
    return 0;
}

/*
 * Adjoint of the 1D forward with the discrete choices (the drift path and the best
 * harmonic count h*) held fixed -- a subgradient through the max of Eq. 2:
 *   dL/dx[j] = sum over (n, k <= h*(n)) with b_k(n) = j of g[n] / sigma[h*(n) - 1],
 * where b_k(n) = k n (simple) or k n + popcount(path[n] & ((1 << k) - 1)) (greedy).
 * form: 1 = simple, 2 = greedy.  grad_x has n entries and is overwritten.
 */
int hso_backward_1d(int32_t form, int64_t n, int32_t H, int64_t nf, const uint8_t *best_h,
                    const uint32_t *path, const double *sigma, const double *g, double *grad_x)
{
    if (!best_h || !sigma || !g || !grad_x || H < 1 || H > HSO_MAX_H) return -1;
    if (form != 1 && form != 2) return -1;
    if (form == 2 && !path) return -1;
    /* nf may reach N - 1 (the truncated tail): every chosen bin must then lie in the spectrum */
    if (nf > n - 1) return -1;
    memset(grad_x, 0, sizeof(double) * (size_t)n);
    for (int64_t f = 0; f < nf; ++f) {
        int hb = best_h[f];
        if (hb < 1 || hb > H) return -1;
        double c = g[f] / sigma[hb - 1];
        for (int k = 1; k <= hb; ++k) {
            int64_t j = (int64_t)k * f;
            if (form == 2) {
                uint32_t mask = (k >= 32) ? 0xffffffffu : ((1u << k) - 1u);
                j += __builtin_popcount(path[f] & mask);
            }
            if (j >= n) return -1;
            grad_x[j] += c;
        }
    }
    return 0;
}

/*
 * Optimal partial sums over every monotone drift path (the "optimal partial sum" the
 * greedy choice approximates, Sec. 3): the chosen drift D_k at order k satisfies
 * D_k - D_{k-1} in {0, 1} (Sec. 2.2), D_0 = 0, D_1 = 0 without mitigation.  Dynamic
 * programme best[k][D] = x[k n + D] + max(best[k-1][D], best[k-1][D-1]);
 * best_sum[h-1] = max_D best[h][D].
 */
int hso_dp_1d(const float *p, const float *w, int32_t round_w, int64_t n, int32_t H,
              int32_t mitigation, int64_t fund, double *best_sum)
{
    if (!p || !best_sum || H < 1 || H > HSO_MAX_H || fund < 0 || fund >= hso_nf_1d(n, H)) return -1;
    double prev[HSO_MAX_H + 2], cur[HSO_MAX_H + 2];
    const double NEG = -INFINITY;
    for (int i = 0; i < HSO_MAX_H + 2; ++i) prev[i] = cur[i] = NEG;
    /* order 1 */
    prev[0] = load_x(p, w, round_w, fund);
    if (mitigation) prev[1] = load_x(p, w, round_w, fund + 1);
    best_sum[0] = prev[0] > prev[1] ? prev[0] : prev[1];
    int dmax = mitigation ? 1 : 0;
    for (int k = 2; k <= H; ++k) {
        int nd = dmax + 1;
        double mx = NEG;
        for (int D = 0; D <= nd; ++D) {
            double stay = (D <= dmax) ? prev[D] : NEG;
            double step = (D >= 1) ? prev[D - 1] : NEG;
            double b = stay > step ? stay : step;
            cur[D] = (b == NEG) ? NEG : b + load_x(p, w, round_w, (int64_t)k * fund + D);
            if (cur[D] > mx) mx = cur[D];
        }
        best_sum[k - 1] = mx;
        dmax = nd;
        for (int D = 0; D <= dmax; ++D) prev[D] = cur[D];
    }
    return 0;
}

/*
 * The optimal form over a spectrum: for every fundamental n < nf the optimal partial sums
 * S*_h (hso_dp_1d above), their SNR by Eq. 2 and its maximum over h = 1..H, starting at h = 1
 * and replaced only by a strictly larger value.  snr_all [nf][H] (may be NULL) receives every
 * order's SNR.
 */
int hso_optimal_1d(const float *p, const float *w, int32_t round_w, int64_t n, int32_t H,
                   int32_t mitigation, const double *mu, const double *sigma, int64_t nf, double *snr,
                   uint8_t *best_h, double *snr_all)
{
    if (!p || !mu || !sigma || !snr || !best_h || H < 1 || H > HSO_MAX_H || nf < 0 || nf > hso_nf_1d(n, H))
        return -1;
    double sums[HSO_MAX_H];
    for (int64_t f = 0; f < nf; ++f) {
        if (hso_dp_1d(p, w, round_w, n, H, mitigation, f, sums) != 0) return -1;
        double best = snr_of(sums[0], 1, mu, sigma);
        int bh = 1;
        for (int h = 1; h <= H; ++h) {
            const double v = snr_of(sums[h - 1], h, mu, sigma);
            if (snr_all) snr_all[f * H + (h - 1)] = v;
            if (h > 1 && v > best) {
                best = v;
                bh = h;
            }
        }
        snr[f] = best;
        best_h[f] = (uint8_t)bh;
    }
    return 0;
}

/*
 * Exhaustive enumeration of all increment sequences b_1..b_H (b_1 = 0 without
 * mitigation): for each h, best_sum[h-1] = max over sequences of sum_{k<=h} x[k n + D_k].
 * It also counts the sequences consistent with the greedy rule at every order
 * (b_k = [x[m+1] > x[m]] with m = k n + D_{k-1}); rule_path receives the last one found.
 * Intended for H <= 20.
 */
int hso_brute_1d(const float *p, const float *w, int32_t round_w, int64_t n, int32_t H,
                 int32_t mitigation, int64_t fund, double *best_sum, uint32_t *rule_path,
                 int64_t *rule_count)
{
    if (!p || !best_sum || H < 1 || H > 20 || fund < 0 || fund >= hso_nf_1d(n, H)) return -1;
    for (int h = 0; h < H; ++h) best_sum[h] = -INFINITY;
    int64_t count = 0;
    uint32_t last = 0;
    const uint32_t nseq = 1u << H;
    for (uint32_t s = 0; s < nseq; ++s) {
        if (!mitigation && (s & 1u)) continue;
        int64_t D = 0;
        double sum = 0.0;
        int consistent = 1;
        for (int k = 1; k <= H; ++k) {
            int64_t m = (int64_t)k * fund + D;      /* candidate pair before the choice */
            int inc = (int)((s >> (k - 1)) & 1u);
            int rule_inc;
            if (k == 1 && !mitigation) rule_inc = 0;
            else rule_inc = load_x(p, w, round_w, m + 1) > load_x(p, w, round_w, m);
            if (inc != rule_inc) consistent = 0;
            D += inc;
            sum += load_x(p, w, round_w, (int64_t)k * fund + D);
            if (sum > best_sum[k - 1]) best_sum[k - 1] = sum;
        }
        if (consistent) { ++count; last = s; }
    }
    if (rule_path) *rule_path = last;
    if (rule_count) *rule_count = count;
    return 0;
}

/*
 * Exhaustive 2D enumeration for one (f, z): all 9^H offset sequences.  best_sum[h-1] is
 * the maximum partial sum of h terms; rule_count counts the sequences whose every step
 * is the strict raster-order maximum with the centre preferred (the 2D greedy rule).
 * Intended for H <= 5.
 */
int hso_brute_2d(const float *plane, int64_t n_freq, int64_t n_rows, int64_t z0_row, int32_t H,
                 int64_t f, int64_t z, double *best_sum, uint32_t *rule_path, int64_t *rule_count)
{
    if (!plane || !best_sum || H < 1 || H > 5) return -1;
    if (f < 1 || (int64_t)H * f + H > n_freq - 1) return -1;
    if (z0_row + (int64_t)H * z - H < 0 || z0_row + (int64_t)H * z + H > n_rows - 1) return -1;
    if (z0_row + z - 1 < 0 || z0_row + z + 1 > n_rows - 1) return -1;
    for (int h = 0; h < H; ++h) best_sum[h] = -INFINITY;
    int64_t total = 1;
    for (int h = 0; h < H; ++h) total *= 9;
    int64_t count = 0;
    uint32_t last = 0;
    for (int64_t s = 0; s < total; ++s) {
        int64_t t = s, df = 0, dz = 0;
        double sum = 0.0;
        int consistent = 1;
        uint32_t bits = 0;
        for (int h = 1; h <= H; ++h) {
            int code = (int)(t % 9);
            t /= 9;
            int of = code % 3 - 1, oz = code / 3 - 1;
            int64_t cf = (int64_t)h * f + df, cr = z0_row + (int64_t)h * z + dz;
            /* the greedy rule's choice at this node */
            double v = (double)plane[cr * n_freq + cf];
            int rcode = 4;
            for (int a = -1; a <= 1; ++a)
                for (int b = -1; b <= 1; ++b) {
                    if (a == 0 && b == 0) continue;
                    double c = (double)plane[(cr + a) * n_freq + (cf + b)];
                    if (c > v) { v = c; rcode = (a + 1) * 3 + (b + 1); }
                }
            if (rcode != code) consistent = 0;
            sum += (double)plane[(cr + oz) * n_freq + (cf + of)];
            if (sum > best_sum[h - 1]) best_sum[h - 1] = sum;
            df += of;
            dz += oz;
            bits |= (uint32_t)code << (4 * (h - 1));
        }
        if (consistent) { ++count; last = bits; }
    }
    if (rule_path) *rule_path = last;
    if (rule_count) *rule_count = count;
    return 0;
}

/*
 * Number of distinct 32-byte sectors of a spectrum of elem_bytes-wide values read by the
 * 1D forms in `forms` (bit 0 simple, bit 1 greedy) over fundamentals [0, nf): the
 * compulsory input footprint.  path = the greedy drift paths (needed when bit 1 is set).
 */
int64_t hso_sectors_1d(int32_t forms, int32_t elem_bytes, int64_t n, int32_t H,
                       int32_t mitigation, int64_t nf, const uint32_t *path)
{
    if (elem_bytes <= 0 || elem_bytes > 32 || H < 1 || H > HSO_MAX_H) return -1;
    if ((forms & 2) && !path) return -1;
    const int64_t per = 32 / elem_bytes;
    const int64_t ns = (n + per - 1) / per;
    uint8_t *seen = (uint8_t *)calloc((size_t)((ns + 7) / 8), 1);
    if (!seen) return -1;
    int64_t count = 0;
#define MARK(j) do { int64_t s_ = (j) / per; \
        if (!(seen[s_ >> 3] & (1u << (s_ & 7)))) { seen[s_ >> 3] |= (uint8_t)(1u << (s_ & 7)); ++count; } } while (0)
    for (int64_t f = 0; f < nf; ++f) {
        if (forms & 1)
            for (int h = 1; h <= H; ++h) MARK((int64_t)h * f);
        if (forms & 2) {
            int64_t d = 0;
            MARK(f);
            if (mitigation) { MARK(f + 1); d = path[f] & 1u; }
            for (int h = 2; h <= H; ++h) {
                int64_t m = (int64_t)h * f + d;
                MARK(m);
                MARK(m + 1);
                d += (path[f] >> (h - 1)) & 1u;
            }
        }
    }
#undef MARK
    free(seen);
    return count;
}

/*
 * Distinct 32-byte sectors of the float32 plane read by the 2D greedy form over the domain
 * [f_lo, f_hi] x [z_lo, z_hi]: the 3x3 neighbourhood of every order along the recorded paths
 * (path[o], 4 bits per order, output index o as in hso_greedy_2d).
 */
int64_t hso_sectors_2d(int64_t n_freq, int64_t n_rows, int64_t z0_row, int32_t H, int64_t f_lo, int64_t f_hi,
                       int64_t z_lo, int64_t z_hi, const uint32_t *path)
{
    if (!path || H < 1 || H > 8 || f_lo < 1 || f_hi < f_lo || z_hi < z_lo) return -1;
    const int64_t per_row = (n_freq + 7) / 8;
    const int64_t ns = per_row * n_rows;
    uint8_t *seen = (uint8_t *)calloc((size_t)((ns + 7) / 8), 1);
    if (!seen) return -1;
    int64_t count = 0;
    const int64_t nff = f_hi - f_lo + 1;
    for (int64_t z = z_lo; z <= z_hi; ++z)
        for (int64_t f = f_lo; f <= f_hi; ++f) {
            const uint32_t bits = path[(z - z_lo) * nff + (f - f_lo)];
            int64_t df = 0, dz = 0;
            for (int h = 1; h <= H; ++h) {
                const int64_t cf = (int64_t)h * f + df, cr = z0_row + (int64_t)h * z + dz;
                for (int oz = -1; oz <= 1; ++oz)
                    for (int of = -1; of <= 1; ++of) {
                        const int64_t s_ = (cr + oz) * per_row + (cf + of) / 8;
                        if (!(seen[s_ >> 3] & (1u << (s_ & 7)))) { seen[s_ >> 3] |= (uint8_t)(1u << (s_ & 7)); ++count; }
                    }
                const int code = (int)((bits >> (4 * (h - 1))) & 0xFu);
                df += code % 3 - 1;
                dz += code / 3 - 1;
            }
        }
    free(seen);
    return count;
}
