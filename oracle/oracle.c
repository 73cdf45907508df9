/*
 * Reference oracle for Branch-and-Bound Tensor Networks (arXiv 2602.05470).
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, obviously-correct CPU
 * restatement of what the GPU path computes. It shares no code with the CUDA
 * library and is used only by the test-suite, the smoke check and the CPU
 * baseline of the benchmark. The product path never calls it.
 *
 * What it computes (all exact integer arithmetic, counts as big integers):
 *
 *  1. Spin-glass ground state by brute force.  Paper Eq. (1):
 *       H(s) = sum_{(i,j) in E} -J_ij s_i s_j + sum_i -h_i s_i ,  s_i in {-1,+1}.
 *     Fields enter as h2 = 2h, so the oracle works with E2 = 2H (integral):
 *       E2(s) = sum_E -2 J_ij s_i s_j + sum_V -h2_i s_i.
 *     Returns min E2 and the number of minimisers (the degeneracy).
 *
 *  2. Maximum-weight independent set by brute force (paper, MWIS paragraph
 *     after Eq. (2)): alpha = max sum_{i in S} w_i over independent sets S, and
 *     the number of sets attaining it.
 *
 *  3. Square-lattice transfer matrix: the same quantity as 1 on an open L x Lc
 *     lattice by a site-by-site sweep whose state is the spins of the last Lc
 *     sites (min over the dropped spin, counts of ties added).  Optional
 *     traceback of one minimiser.
 *
 *  4. King's-subgraph transfer matrix: the same quantity as 2 on a site mask of
 *     an N x Nc grid with king-move adjacency; the state is the occupation of
 *     the last Nc+1 sites, kept as a sorted sparse list of independent masks.
 *
 *  5. One counting-tropical pairwise contraction by its definition (paper
 *     Eq. (2) with the counting algebra of the paragraph that follows it):
 *     every entry of C is (max over the summed indices of A + B, sum over the
 *     maximising assignments of cA*cB mod p) -- max-plus form of the min-sum
 *     algebra, values floored at the -infinity sentinel `neg`.
 *
 * Counts in 3 and 4 are fixed-width little-endian big integers of `w64` 64-bit
 * limbs; on carry out of the top limb the routine returns ORACLE_OVERFLOW and
 * the caller retries with more limbs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_OVERFLOW (-3)

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- bignums */

/* dst += src (w limbs); returns the carry out of the top limb */
static int big_add(uint64_t *dst, const uint64_t *src, int w) {
    uint64_t carry = 0;
    for (int i = 0; i < w; i++) {
        u128 s = (u128)dst[i] + src[i] + carry;
        dst[i] = (uint64_t)s;
        carry = (uint64_t)(s >> 64);
    }
    return carry != 0;
}

/* decimal text of a w-limb number; returns length or -1 if cap too small */
static int big_to_dec(const uint64_t *x, int w, char *out, size_t cap) {
    uint64_t *t = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(w > 0 ? w : 1));
    if (!t) return -1;
    memcpy(t, x, sizeof(uint64_t) * (size_t)w);
    char buf[4096 * 2];
    int n = 0;
    const uint64_t base = 1000000000000000000ull; /* 10^18 */
    for (;;) {
        int nz = 0;
        for (int i = 0; i < w; i++) if (t[i]) { nz = 1; break; }
        if (!nz) break;
        u128 rem = 0;
        for (int i = w - 1; i >= 0; i--) {
            u128 cur = (rem << 64) | t[i];
            t[i] = (uint64_t)(cur / base);
            rem = cur % base;
        }
        uint64_t r = (uint64_t)rem;
        for (int k = 0; k < 18; k++) {
            if ((size_t)n >= sizeof(buf)) { free(t); return -1; }
            buf[n++] = (char)('0' + (int)(r % 10));
            r /= 10;
        }
    }
    free(t);
    while (n > 1 && buf[n - 1] == '0') n--;
    if (n == 0) buf[n++] = '0';
    if ((size_t)n + 1 > cap) return -1;
    for (int i = 0; i < n; i++) out[i] = buf[n - 1 - i];
    out[n] = 0;
    return n;
}

/* ------------------------------------------------------ 1. spin brute force */

int oracle_spin_bruteforce(int n, int m, const int32_t *edges, const int32_t *J,
                           const int32_t *h2, int64_t *e2_out, uint64_t *count_out,
                           int8_t *config_out) {
    if (n < 0 || n > 34 || m < 0) return ORACLE_EINVAL;
    int64_t best = INT64_MAX;
    uint64_t cnt = 0, best_cfg = 0;
    uint64_t total = 1ull << n;
    for (uint64_t cfg = 0; cfg < total; cfg++) {
        int64_t e = 0;
        for (int k = 0; k < m; k++) {
            int i = edges[2 * k], j = edges[2 * k + 1];
            int si = ((cfg >> i) & 1) ? 1 : -1, sj = ((cfg >> j) & 1) ? 1 : -1;
            e += -2LL * J[k] * si * sj;
        }
        if (h2)
            for (int i = 0; i < n; i++) e += -(int64_t)h2[i] * (((cfg >> i) & 1) ? 1 : -1);
        if (e < best) { best = e; cnt = 1; best_cfg = cfg; }
        else if (e == best) cnt++;
    }
    *e2_out = best;
    *count_out = cnt;
    if (config_out)
        for (int i = 0; i < n; i++) config_out[i] = ((best_cfg >> i) & 1) ? 1 : -1;
    return ORACLE_OK;
}

/* ------------------------------------------------------ 2. MWIS brute force */

int oracle_mwis_bruteforce(int n, int m, const int32_t *edges, const int32_t *w,
                           int64_t *best_out, uint64_t *count_out, int8_t *config_out) {
    if (n < 0 || n > 34 || m < 0) return ORACLE_EINVAL;
    int64_t best = -1;
    uint64_t cnt = 0, best_cfg = 0;
    uint64_t total = 1ull << n;
    for (uint64_t cfg = 0; cfg < total; cfg++) {
        int ok = 1;
        for (int k = 0; k < m && ok; k++)
            if (((cfg >> edges[2 * k]) & 1) && ((cfg >> edges[2 * k + 1]) & 1)) ok = 0;
        if (!ok) continue;
        int64_t s = 0;
        for (int i = 0; i < n; i++) if ((cfg >> i) & 1) s += w ? w[i] : 1;
        if (s > best) { best = s; cnt = 1; best_cfg = cfg; }
        else if (s == best) cnt++;
    }
    *best_out = best;
    *count_out = cnt;
    if (config_out)
        for (int i = 0; i < n; i++) config_out[i] = (int8_t)((best_cfg >> i) & 1);
    return ORACLE_OK;
}

/* ------------------------------------------ 3. square-lattice transfer matrix */
/*
 * Sites t = r*Lc + c in row-major order. After site t the state holds the
 * spins of sites t-Lc+1 .. t (bit 0 = oldest, bit Lc-1 = newest; bit set means
 * spin +1). Adding site t (row r >= 1) couples it to site t-Lc (bit 0, the
 * site above, which leaves the window) and to site t-1 (bit Lc-1) when c > 0.
 * Jh[r*(Lc-1)+c] couples (r,c)-(r,c+1); Jv[r*Lc+c] couples (r,c)-(r+1,c).
 */
int oracle_spin_square_tm(int L, int Lc, const int32_t *Jh, const int32_t *Jv,
                          const int32_t *h2, int w64, int64_t *e2_out, char *count_dec,
                          size_t dec_cap, int8_t *config_out) {
    if (L < 1 || Lc < 1 || Lc > 26 || w64 < 1) return ORACLE_EINVAL;
    const uint64_t S = 1ull << Lc;
    int64_t *val = (int64_t *)malloc(sizeof(int64_t) * S);
    int64_t *nval = (int64_t *)malloc(sizeof(int64_t) * S);
    uint64_t *cnt = (uint64_t *)calloc(S * (size_t)w64, sizeof(uint64_t));
    uint64_t *ncnt = (uint64_t *)calloc(S * (size_t)w64, sizeof(uint64_t));
    uint8_t *choice = NULL;     /* choice[(t-Lc)*S + mask]: which dropped spin won */
    const int nsites = L * Lc;
    if (config_out && L > 1) choice = (uint8_t *)malloc((size_t)(nsites - Lc) * S);
    if (!val || !nval || !cnt || !ncnt || (config_out && L > 1 && !choice)) {
        free(val); free(nval); free(cnt); free(ncnt); free(choice);
        return ORACLE_ENOMEM;
    }
    int rc = ORACLE_OK;
    /* first row: enumerate all of its spins directly */
    for (uint64_t mask = 0; mask < S; mask++) {
        int64_t e = 0;
        for (int c = 0; c < Lc; c++) {
            int sc = ((mask >> c) & 1) ? 1 : -1;
            e += -(int64_t)(h2 ? h2[c] : 0) * sc;
            if (c + 1 < Lc) {
                int sn = ((mask >> (c + 1)) & 1) ? 1 : -1;
                e += -2LL * Jh[c] * sc * sn;
            }
        }
        val[mask] = e;
        cnt[mask * w64] = 1;
    }
    for (int t = Lc; t < nsites && rc == ORACLE_OK; t++) {
        int r = t / Lc, c = t % Lc;
        int32_t jv = Jv[(r - 1) * Lc + c];
        int32_t jh = (c > 0) ? Jh[r * (Lc - 1) + (c - 1)] : 0;
        int32_t hf = h2 ? h2[t] : 0;
        for (uint64_t nm = 0; nm < S; nm++) {
            int st = (int)((nm >> (Lc - 1)) & 1);
            int sig = st ? 1 : -1;
            uint64_t base = (nm << 1) & (S - 1);
            int64_t bestv = INT64_MAX;
            int bestb = 0;
            int64_t cand[2];
            for (int b = 0; b < 2; b++) {
                uint64_t m = base | (uint64_t)b;
                int sup = b ? 1 : -1;                      /* spin above (bit 0) */
                int sleft = ((m >> (Lc - 1)) & 1) ? 1 : -1; /* spin to the left */
                int64_t e = val[m] - 2LL * jv * sup * sig - (int64_t)hf * sig;
                if (c > 0) e += -2LL * jh * sleft * sig;
                cand[b] = e;
                if (e < bestv) { bestv = e; bestb = b; }
            }
            nval[nm] = bestv;
            uint64_t *dst = ncnt + nm * w64;
            memset(dst, 0, sizeof(uint64_t) * (size_t)w64);
            for (int b = 0; b < 2; b++)
                if (cand[b] == bestv && big_add(dst, cnt + (base | (uint64_t)b) * w64, w64))
                    rc = ORACLE_OVERFLOW;
            if (choice) choice[(size_t)(t - Lc) * S + nm] = (uint8_t)bestb;
        }
        int64_t *tv = val; val = nval; nval = tv;
        uint64_t *tc = cnt; cnt = ncnt; ncnt = tc;
    }
    if (rc == ORACLE_OK) {
        int64_t best = INT64_MAX;
        uint64_t bestmask = 0;
        for (uint64_t m = 0; m < S; m++) if (val[m] < best) { best = val[m]; bestmask = m; }
        uint64_t *tot = (uint64_t *)calloc((size_t)w64, sizeof(uint64_t));
        for (uint64_t m = 0; m < S && rc == ORACLE_OK; m++)
            if (val[m] == best && big_add(tot, cnt + m * w64, w64)) rc = ORACLE_OVERFLOW;
        *e2_out = best;
        if (rc == ORACLE_OK && count_dec && big_to_dec(tot, w64, count_dec, dec_cap) < 0)
            rc = ORACLE_EINVAL;
        free(tot);
        if (rc == ORACLE_OK && config_out) {
            uint64_t mask = bestmask;
            for (int t = nsites - 1; t >= Lc; t--) {
                config_out[t] = ((mask >> (Lc - 1)) & 1) ? 1 : -1;
                uint64_t b = choice[(size_t)(t - Lc) * S + mask];
                mask = ((mask << 1) & (S - 1)) | b;
            }
            for (int c = 0; c < Lc; c++) config_out[c] = ((mask >> c) & 1) ? 1 : -1;
        }
    }
    free(val); free(nval); free(cnt); free(ncnt); free(choice);
    return rc;
}

/* --------------------------------------------- 4. King's-subgraph transfer matrix */
/*
 * Sites t = r*Nc + c. Before site t the state holds the occupation of sites
 * t-Nc-1 .. t-1 (bit j <-> site t-Nc-1+j): bit 0 = up-left, bit 1 = up,
 * bit 2 = up-right, bit Nc = left. The oldest site leaves the window after t.
 * States are kept as a list sorted by mask; the shift m >> 1 keeps that order and
 * makes the two states that differ only in the dropped site adjacent.
 */
typedef struct { uint64_t mask; int64_t val; } tm_key;

int oracle_mwis_ksg_tm(int N, int Nc, const uint8_t *site, const int32_t *w, int w64,
                       int64_t *best_out, char *count_dec, size_t dec_cap,
                       uint64_t *max_states_out) {
    if (N < 1 || Nc < 1 || Nc > 60 || w64 < 1) return ORACLE_EINVAL;
    size_t capn = 1024;
    size_t ns = 1;
    tm_key *st = (tm_key *)malloc(sizeof(tm_key) * capn);
    uint64_t *sc = (uint64_t *)calloc(capn * (size_t)w64, sizeof(uint64_t));
    if (!st || !sc) { free(st); free(sc); return ORACLE_ENOMEM; }
    st[0].mask = 0; st[0].val = 0; sc[0] = 1;
    uint64_t maxst = 1;
    int rc = ORACLE_OK;
    const uint64_t top = 1ull << Nc;
    for (int t = 0; t < N * Nc && rc == ORACLE_OK; t++) {
        int r = t / Nc, c = t % Nc;
        int present = site[t] != 0;
        uint64_t nb = 0;
        if (c > 0) nb |= top;                 /* left */
        if (r > 0 && c > 0) nb |= 1;          /* up-left */
        if (r > 0) nb |= 2;                   /* up */
        if (r > 0 && c + 1 < Nc) nb |= 4;     /* up-right */
        int64_t wt = w ? w[t] : 1;
        size_t ncap = 2 * ns + 2;
        tm_key *nst = (tm_key *)malloc(sizeof(tm_key) * ncap);
        uint64_t *nsc = (uint64_t *)calloc(ncap * (size_t)w64, sizeof(uint64_t));
        if (!nst || !nsc) { free(nst); free(nsc); rc = ORACLE_ENOMEM; break; }
        size_t nn = 0;
        for (int x = 0; x < 2; x++) {
            if (x == 1 && !present) break;
            for (size_t i = 0; i < ns; i++) {
                if (x == 1 && (st[i].mask & nb)) continue;
                uint64_t nm = (st[i].mask >> 1) | (x ? top : 0);
                int64_t v = st[i].val + (x ? wt : 0);
                if (nn > 0 && nst[nn - 1].mask == nm) {
                    uint64_t *dst = nsc + (nn - 1) * w64;
                    if (v > nst[nn - 1].val) {
                        nst[nn - 1].val = v;
                        memcpy(dst, sc + i * w64, sizeof(uint64_t) * (size_t)w64);
                    } else if (v == nst[nn - 1].val) {
                        if (big_add(dst, sc + i * w64, w64)) rc = ORACLE_OVERFLOW;
                    }
                } else {
                    nst[nn].mask = nm;
                    nst[nn].val = v;
                    memcpy(nsc + nn * w64, sc + i * w64, sizeof(uint64_t) * (size_t)w64);
                    nn++;
                }
            }
        }
        free(st); free(sc);
        st = nst; sc = nsc; ns = nn;
        if (ns > maxst) maxst = ns;
    }
    if (rc == ORACLE_OK) {
        int64_t best = INT64_MIN;
        for (size_t i = 0; i < ns; i++) if (st[i].val > best) best = st[i].val;
        uint64_t *tot = (uint64_t *)calloc((size_t)w64, sizeof(uint64_t));
        for (size_t i = 0; i < ns && rc == ORACLE_OK; i++)
            if (st[i].val == best && big_add(tot, sc + i * w64, w64)) rc = ORACLE_OVERFLOW;
        *best_out = best;
        if (rc == ORACLE_OK && count_dec && big_to_dec(tot, w64, count_dec, dec_cap) < 0)
            rc = ORACLE_EINVAL;
        free(tot);
    }
    if (max_states_out) *max_states_out = maxst;
    free(st); free(sc);
    return rc;
}

/* ---------------------------------- 5. counting-tropical pairwise contraction */
/*
 * Tensors over binary variables. Bit i of a tensor's linear index is the value
 * of variable labels[i]. A value plane (int32) and np count planes (residues
 * mod primes[t], plane t at offset t * 2^r) per tensor.
 *
 *   C[lc] = max( neg , max_{s} A[la] + B[lb] )        s = (la U lb) \ lc
 *   cC_t[lc] = sum_{s attaining the max} cA_t * cB_t   mod primes[t]
 *
 * A label appearing in C must appear in A or B. rb = -1 means "no B" (the
 * single-operand reduction: B is the scalar with value 0 and count 1).
 */
static int find_label(int r, const int32_t *l, int32_t x) {
    for (int i = 0; i < r; i++) if (l[i] == x) return i;
    return -1;
}

int oracle_contract(int ra, const int32_t *la, const int32_t *va, const uint64_t *ca,
                    int rb, const int32_t *lb, const int32_t *vb, const uint64_t *cb,
                    int rc, const int32_t *lc, int32_t *vc, uint64_t *cc,
                    int np, const uint64_t *primes, int32_t neg) {
    if (ra < 0 || rc < 0 || rb < -1 || np < 0 || ra > 30 || rb > 30 || rc > 30) return ORACLE_EINVAL;
    int rbb = rb < 0 ? 0 : rb;
    /* union of labels: C's first, then the summed ones */
    int32_t u[96];
    int nu = 0;
    for (int i = 0; i < rc; i++) {
        if (find_label(ra, la, lc[i]) < 0 && find_label(rbb, lb, lc[i]) < 0) return ORACLE_EINVAL;
        u[nu++] = lc[i];
    }
    for (int i = 0; i < ra; i++) if (find_label(nu, u, la[i]) < 0) u[nu++] = la[i];
    for (int i = 0; i < rbb; i++) if (find_label(nu, u, lb[i]) < 0) u[nu++] = lb[i];
    int ns = nu - rc;
    if (ns > 30) return ORACLE_EINVAL;
    int posA[96], posB[96];
    for (int i = 0; i < nu; i++) { posA[i] = find_label(ra, la, u[i]); posB[i] = find_label(rbb, lb, u[i]); }
    const uint64_t nout = 1ull << rc, nsum = 1ull << ns;
    const uint64_t sizeA = 1ull << ra, sizeB = 1ull << rbb;
    for (uint64_t o = 0; o < nout; o++) {
        /* pass 1: the maximum */
        int32_t best = neg;
        for (uint64_t s = 0; s < nsum; s++) {
            uint64_t full = o | (s << rc);
            uint64_t ia = 0, ib = 0;
            for (int i = 0; i < nu; i++) {
                uint64_t bit = (full >> i) & 1;
                if (posA[i] >= 0) ia |= bit << posA[i];
                if (posB[i] >= 0) ib |= bit << posB[i];
            }
            int64_t v = (int64_t)va[ia] + (rb >= 0 ? (int64_t)vb[ib] : 0);
            if (v > best) best = (int32_t)v;
        }
        vc[o] = best;
        /* pass 2: counts of the maximising assignments */
        for (int t = 0; t < np; t++) {
            uint64_t p = primes[t];
            uint64_t acc = 0;
            for (uint64_t s = 0; s < nsum; s++) {
                uint64_t full = o | (s << rc);
                uint64_t ia = 0, ib = 0;
                for (int i = 0; i < nu; i++) {
                    uint64_t bit = (full >> i) & 1;
                    if (posA[i] >= 0) ia |= bit << posA[i];
                    if (posB[i] >= 0) ib |= bit << posB[i];
                }
                int64_t v = (int64_t)va[ia] + (rb >= 0 ? (int64_t)vb[ib] : 0);
                if (v != best) continue;
                uint64_t x = ca[(size_t)t * sizeA + ia] % p;
                uint64_t y = rb >= 0 ? cb[(size_t)t * sizeB + ib] % p : 1;
                acc = (uint64_t)(((u128)acc + (u128)x * y) % p);
            }
            cc[(size_t)t * nout + o] = acc;
        }
    }
    return ORACLE_OK;
}
