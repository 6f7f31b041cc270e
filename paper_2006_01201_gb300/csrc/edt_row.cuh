// edt_row.cuh -- internal: the per-thread steps of the row pass of the exact
// distance transform behind Eq. (1) (edt.cu). Host and device functions on
// plain arrays (device functions under nvcc, plain inline functions under a
// host compiler); the kernel in edt.cu orders them with barriers and scans.
//
// Row pass, for one area (Area1 or Area2) and one canvas row: the squared
// distance at column x is
//   d2(x) = min over sites q of (x - q)^2 + f(q),   f(q) = g(q)^2,
// g(q) the vertical distance of column q to its nearest feature pixel
// (columns without one are no site). The minimum is the lower envelope of
// one parabola per site (Felzenszwalb & Huttenlocher, "Distance transforms
// of sampled functions", 2012). The row is cut into bands of consecutive
// columns, one per thread:
//   1. each thread builds the envelope of its band's sites (a stack);
//   2. groups of bands are merged pairwise in a tree. The envelope of two
//      groups, all sites of the left one left of the right one's, keeps a
//      prefix of the left envelope and a suffix of the right one (the
//      banding idea of Cao, Tang, Mukherjee & Lee, "Parallel Banding
//      Algorithm to compute exact distance transform with the GPU", 2010):
//      one thread pushes the right envelope's sites onto the left one,
//      popping hidden sites, until a right site lands on another right
//      site, after which nothing more changes;
//   3. each band's first kept site gets the integer start of its region,
//      and a thread reads its own columns by a walk from the site that owns
//      the first of them.
// The intersection abscissae of two parabolas are rationals; they are
// compared by cross-multiplication in 64-bit integers, so d2 is exact.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define PANO_HD __device__ __forceinline__
#else
#define PANO_HD inline
#endif

#ifndef PANO_AT
#include "bounds.cuh"
#endif

namespace pano {
namespace edt {

constexpr uint32_t kNoSite = 0xFFFFu;  // g of a column without a feature pixel of the area

// g of column q of the row of one area
PANO_HD uint32_t g_of(const uint16_t* gs, int w, int q) { return PANO_AT(gs, q, w, 520); }

PANO_HD long long f_of(const uint16_t* gs, int w, int q) {
    const long long v = g_of(gs, w, q);
    return v * v;
}

// abscissa where the parabolas of sites p < q meet: num / den, den > 0
PANO_HD void meet(long long fp, int p, long long fq, int q, long long* num, long long* den) {
    *num = (fq + (long long)q * q) - (fp + (long long)p * p);
    *den = 2LL * (q - p);
}

// the parabola of b (a < b < q) has no part of the envelope of a, b, q:
// s(b, q) <= s(a, b)
PANO_HD bool hidden(long long fa, int a, long long fb, int b, long long fq, int q) {
    long long n0, d0, n1, d1;
    meet(fa, a, fb, b, &n0, &d0);
    meet(fb, b, fq, q, &n1, &d1);
    return n1 * d0 <= n0 * d1;
}

// q owns column x against p < q: x >= s(p, q)
PANO_HD bool owns(long long fp, int p, long long fq, int q, int x) {
    long long n, d;
    meet(fp, p, fq, q, &n, &d);
    return n <= (long long)x * d;
}

// Step 0 (optional, changes no d2): sites that two other sites hide have
// no part of the envelope of the whole row, so they can be dropped before
// it is built. Here g is often a staircase of plateaus (equal g over many
// columns), and the first columns of a higher plateau are hidden by the
// last column of the lower plateau before it and their right neighbour.
// Inside a band the band envelope drops them; at a band's edges the merges
// would pop them one by one. So each thread tests the run of equal g that
// its band starts with against the column L before that run (if its g is
// smaller), and the run it ends with against the column R after that run.
// Marks the dropped columns of [x0, x1) with 1 in flag[] (0 elsewhere).
PANO_HD void edge_runs_hidden(const uint16_t* gs, uint16_t* flag, int w, int x0, int x1, int L, int R) {
    for (int q = x0; q < x1; ++q) PANO_AT(flag, q, w, 545) = 0;
    if (x0 >= x1) return;
    const uint32_t G = g_of(gs, w, x0);
    if (G != kNoSite && G != 0 && L >= 0 && g_of(gs, w, L) < G) {  // kNoSite is no smaller
        const long long fL = f_of(gs, w, L), fG = (long long)G * G;
        for (int q = x0; q < x1 && g_of(gs, w, q) == G; ++q) {
            const int c = q + 1;
            if (c >= w || g_of(gs, w, c) == kNoSite) break;
            if (hidden(fL, L, fG, q, f_of(gs, w, c), c)) flag[q] = 1;
        }
    }
    const uint32_t H = g_of(gs, w, x1 - 1);
    if (H != kNoSite && H != 0 && R < w && g_of(gs, w, R) < H) {
        const long long fR = f_of(gs, w, R), fH = (long long)H * H;
        for (int q = x1 - 1; q >= x0 && g_of(gs, w, q) == H; --q) {
            const int c = q - 1;
            if (c < 0 || g_of(gs, w, c) == kNoSite) break;
            if (hidden(f_of(gs, w, c), c, fH, q, fR, R)) flag[q] = 1;
        }
    }
}

// where runs of equal g begin and end in [x0, x1): the last column c with
// c == 0 or g[c] != g[c-1] (-1 if none) and the first column c with
// c == w-1 or g[c] != g[c+1] (w if none)
PANO_HD void band_run_edges(const uint16_t* gs, int w, int x0, int x1, int* last_start, int* first_end) {
    int ls = -1, fe = w;
    for (int c = x0; c < x1; ++c) {
        if (c == 0 || g_of(gs, w, c) != g_of(gs, w, c - 1)) ls = c;
        if (fe == w && (c == w - 1 || g_of(gs, w, c) != g_of(gs, w, c + 1))) fe = c;
    }
    *last_start = ls;
    *first_end = fe;
}

// Step 1: envelope of the sites of columns [x0, x1), stored at st[x0 ..];
// returns their count. The two top sites and their f stay in registers.
PANO_HD int band_envelope(const uint16_t* gs, uint16_t* st, int w, int x0, int x1) {
    int k = 0;
    int t1 = 0, t2 = 0;  // top and second site (valid for k >= 1, k >= 2)
    long long f1 = 0, f2 = 0;
    for (int q = x0; q < x1; ++q) {
        const uint32_t gq = g_of(gs, w, q);
        if (gq == kNoSite) continue;
        const long long fq = (long long)gq * gq;
        while (k >= 2 && hidden(f2, t2, f1, t1, fq, q)) {
            --k;  // pop t1
            t1 = t2;
            f1 = f2;
            if (k >= 2) {
                t2 = PANO_AT(st, x0 + k - 2, w, 521);
                f2 = f_of(gs, w, t2);
            }
        }
        PANO_AT(st, x0 + k, w, 522) = (uint16_t)q;
        ++k;
        t2 = t1;
        f2 = f1;
        t1 = q;
        f1 = fq;
    }
    return k;
}

// the band before b, not before `first`, that keeps a site; -1 if none
PANO_HD int prev_kept(const int* lo, const int* hi, int nb, int b, int first) {
    for (--b; b >= first; --b)
        if (PANO_AT(hi, b, nb, 523) > PANO_AT(lo, b, nb, 523)) return b;
    return -1;
}

// the band after b, not after `last`, that keeps a site; -1 if none
PANO_HD int next_kept(const int* lo, const int* hi, int nb, int b, int last) {
    for (++b; b <= last; ++b)
        if (PANO_AT(hi, b, nb, 524) > PANO_AT(lo, b, nb, 524)) return b;
    return -1;
}

// Step 2: merge the envelope of the left group (its kept sites in bands
// lf .. ll, both keeping sites) with that of the right group (rf .. rl).
// Band b keeps st[lo[b] .. hi[b]); the merge lowers hi[] at the end of the
// left group and raises lo[] at the start of the right one. The left group
// keeps at least its first site and the right one its last, so the merged
// group runs from lf to rl. The top of the merged stack (the left's last
// site l1 and the right site q being pushed) stays in registers. Returns
// false if the iteration limit (more steps than there are sites, which a
// valid input never needs) was reached.
PANO_HD bool merge_groups(const uint16_t* gs, const uint16_t* st, int* lo, int* hi, int w, int nb, int lf,
                          int ll, int rf, int rl) {
    int lb = ll;  // band of the left's last kept site l1 = st[lhi - 1]
    int llo = PANO_AT(lo, lb, nb, 525), lhi = PANO_AT(hi, lb, nb, 525);
    int l1 = PANO_AT(st, lhi - 1, w, 526);
    long long f1 = f_of(gs, w, l1);
    // the site below l1 (l2 = st[i2] of band pb; pb < 0: l1 is the left's only site), found once
    // and again only after a pop
    int pb = -1, l2 = 0;
    long long f2 = 0;
    bool have2 = false;
    int sb = rf, si = PANO_AT(lo, rf, nb, 527);  // q = st[si] of band sb: the right site being pushed
    int q = PANO_AT(st, si, w, 528);
    long long fq = f_of(gs, w, q);
    bool ok = false;
    for (int it = 0; it <= 2 * w + 2; ++it) {
        // push q: first pop the left sites it hides (the left keeps >= 1)
        for (int pops = 0; pops <= w; ++pops) {
            if (!have2) {
                int i2 = lhi - 2;
                pb = lb;
                if (i2 < llo) {
                    pb = prev_kept(lo, hi, nb, lb, lf);
                    if (pb >= 0) i2 = PANO_AT(hi, pb, nb, 529) - 1;
                }
                if (pb >= 0) {
                    l2 = PANO_AT(st, i2, w, 530);
                    f2 = f_of(gs, w, l2);
                }
                have2 = true;
            }
            if (pb < 0 || !hidden(f2, l2, f1, l1, fq, q)) break;
            if (--lhi == llo) {  // band lb loses its last kept site
                PANO_AT(hi, lb, nb, 531) = lhi;
                lb = pb;
                llo = PANO_AT(lo, lb, nb, 531);
                lhi = PANO_AT(hi, lb, nb, 531);
            }
            l1 = l2;
            f1 = f2;
            have2 = false;
        }
        // q is pushed: the right site after it
        int nbd = sb, ni = si + 1;
        if (ni >= PANO_AT(hi, sb, nb, 532)) {
            nbd = next_kept(lo, hi, nb, sb, rl);
            if (nbd < 0) {
                ok = true;  // every right site processed
                break;
            }
            ni = PANO_AT(lo, nbd, nb, 533);
        }
        const int q2 = PANO_AT(st, ni, w, 534);
        const long long fq2 = f_of(gs, w, q2);
        if (!hidden(f1, l1, fq, q, fq2, q2)) {
            ok = true;  // q2 lands on q: the rest of the right envelope stays
            break;
        }
        sb = nbd;  // q is popped; q2 is pushed next
        si = ni;
        q = q2;
        fq = fq2;
    }
    PANO_AT(hi, lb, nb, 535) = lhi;
    for (int b = rf; b < sb; ++b) PANO_AT(lo, b, nb, 536) = hi[b];  // popped right bands
    PANO_AT(lo, sb, nb, 537) = si;
    return ok;
}

// integer start of the region of site q after p (p < q): the least column x
// with x >= s(p, q), limited to [-1, w] (enough for columns 0 .. w-1)
PANO_HD int region_start(long long fp, int p, long long fq, int q, int w) {
    long long n, d;
    meet(fp, p, fq, q, &n, &d);
    long long z = n >= 0 ? (n + d - 1) / d : -((-n) / d);  // ceil(n / d), d > 0
    if (z < -1) z = -1;
    if (z > w) z = w;
    return (int)z;
}

// Step 3: a walk along the merged envelope; the owner of column x is the
// last kept site whose region starts at or before x. zs[b] is the start of
// band b's first kept site (-1 for the first band with a site); a band with
// no site holds the start of the next band with one (w if none), so zs is
// non-decreasing. nxt[b]: the first band >= b that keeps a site (nb if none).
struct Walker {
    int b, j, hb;  // the owner is st[j] of band b; hb = hi[b]
    int s;         // the owner's column
    long long fs;  // and its f
};

PANO_HD Walker walk_start(const uint16_t* gs, const uint16_t* st, const int* lo, const int* hi, const int* zs, int w,
                          int nb, int x) {
    int l = 0, r = nb - 1;  // largest b with zs[b] <= x (zs[first kept band] = -1)
    while (l < r) {
        const int m = (l + r + 1) >> 1;
        if (PANO_AT(zs, m, nb, 538) <= x) l = m;
        else r = m - 1;
    }
    Walker k;
    k.b = l;
    k.j = PANO_AT(lo, l, nb, 539);
    k.hb = PANO_AT(hi, l, nb, 539);
    k.s = PANO_AT(st, k.j, w, 540);
    k.fs = f_of(gs, w, k.s);
    for (int it = 0; it < w && k.j + 1 < k.hb; ++it) {
        const int q = PANO_AT(st, k.j + 1, w, 541);
        const long long fq = f_of(gs, w, q);
        if (!owns(k.fs, k.s, fq, q, x)) break;
        ++k.j;
        k.s = q;
        k.fs = fq;
    }
    return k;
}

// moves the walker to the owner of column x (x not left of the last one)
// and returns d2(x)
PANO_HD long long walk_to(const uint16_t* gs, const uint16_t* st, const int* lo, const int* hi, const int* nxt, int w,
                          int nb, int x, Walker* k) {
    for (int it = 0; it < w; ++it) {
        int b = k->b, j = k->j + 1, hb = k->hb;
        if (j >= hb) {
            if (b + 1 >= nb) break;
            b = PANO_AT(nxt, b + 1, nb, 542);
            if (b >= nb) break;
            j = PANO_AT(lo, b, nb, 543);
            hb = PANO_AT(hi, b, nb, 543);
        }
        const int q = PANO_AT(st, j, w, 544);
        const long long fq = f_of(gs, w, q);
        if (!owns(k->fs, k->s, fq, q, x)) break;
        k->b = b;
        k->j = j;
        k->hb = hb;
        k->s = q;
        k->fs = fq;
    }
    const long long dx = x - k->s;
    return dx * dx + k->fs;
}

}  // namespace edt
}  // namespace pano
