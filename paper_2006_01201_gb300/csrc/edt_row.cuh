// edt_row.cuh -- internal: the per-thread steps of the row pass of the exact
// distance transform behind Eq. (1) (edt.cu). Host and device functions on
// plain arrays (device functions under nvcc, plain inline functions under a
// host compiler); the kernel in edt.cu orders them with barriers and scans.
//
// Row pass, per area a (0: Area1, 1: Area2) of one canvas row: the squared
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

// g of column q for area a from the packed row (g of Area1 in the low half,
// of Area2 in the high half)
PANO_HD uint32_t g_of(const uint32_t* gs, int w, int a, int q) { return (PANO_AT(gs, q, w, 520) >> (16 * a)) & 0xFFFFu; }

PANO_HD long long f_of(const uint32_t* gs, int w, int a, int q) {
    const long long v = g_of(gs, w, a, q);
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

// Step 1: envelope of the sites of columns [x0, x1), stored at st[x0 ..];
// returns their count.
PANO_HD int band_envelope(const uint32_t* gs, uint16_t* st, int w, int a, int x0, int x1) {
    int k = 0;
    for (int q = x0; q < x1; ++q) {
        if (g_of(gs, w, a, q) == kNoSite) continue;
        const long long fq = f_of(gs, w, a, q);
        while (k >= 2) {
            const int b = PANO_AT(st, x0 + k - 1, w, 521), p = PANO_AT(st, x0 + k - 2, w, 521);
            if (hidden(f_of(gs, w, a, p), p, f_of(gs, w, a, b), b, fq, q)) --k;
            else break;
        }
        PANO_AT(st, x0 + k, w, 522) = (uint16_t)q;
        ++k;
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
// group runs from lf to rl. Returns false if the iteration limit (more steps
// than there are sites, which a valid input never needs) was reached.
PANO_HD bool merge_groups(const uint32_t* gs, const uint16_t* st, int* lo, int* hi, int w, int nb, int a, int lf,
                          int ll, int rf, int rl) {
    int lb = ll;               // band of the left group's last kept site
    int sb = rf, si = PANO_AT(lo, rf, nb, 525);  // first right site still kept: st[si] of band sb
    bool pushed = false;       // st[si] is on the merged stack
    bool ok = false;
    for (int it = 0; it <= 2 * w + 2; ++it) {
        if (!pushed) {
            // push st[si]: first pop the left sites it hides (the left keeps >= 1)
            const int q = PANO_AT(st, si, w, 526);
            const long long fq = f_of(gs, w, a, q);
            for (int pops = 0; pops <= w; ++pops) {
                const int n = PANO_AT(hi, lb, nb, 527) - PANO_AT(lo, lb, nb, 527);
                int l2;
                if (n >= 2) {
                    l2 = PANO_AT(st, hi[lb] - 2, w, 528);
                } else {
                    const int pb = prev_kept(lo, hi, nb, lb, lf);
                    if (pb < 0) break;
                    l2 = PANO_AT(st, hi[pb] - 1, w, 528);
                }
                const int l1 = PANO_AT(st, hi[lb] - 1, w, 529);
                if (!hidden(f_of(gs, w, a, l2), l2, f_of(gs, w, a, l1), l1, fq, q)) break;
                if (--hi[lb] == lo[lb]) lb = prev_kept(lo, hi, nb, lb, lf);
            }
            pushed = true;
            continue;
        }
        // st[si] is pushed: look at the right site after it
        int nbd = sb, ni = si + 1;
        if (ni >= PANO_AT(hi, sb, nb, 530)) {
            nbd = next_kept(lo, hi, nb, sb, rl);
            if (nbd < 0) {
                ok = true;  // every right site processed
                break;
            }
            ni = lo[nbd];
        }
        const int top = PANO_AT(st, si, w, 531), q = PANO_AT(st, ni, w, 531), l1 = PANO_AT(st, hi[lb] - 1, w, 531);
        if (hidden(f_of(gs, w, a, l1), l1, f_of(gs, w, a, top), top, f_of(gs, w, a, q), q)) {
            sb = nbd;  // st[si] is popped; the next right site comes next
            si = ni;
            pushed = false;
        } else {
            ok = true;  // q lands on a right site: the rest of the right envelope stays
            break;
        }
    }
    for (int b = rf; b < sb; ++b) PANO_AT(lo, b, nb, 532) = hi[b];  // popped right bands
    PANO_AT(lo, sb, nb, 533) = si;
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
    int b, j;  // the owner is st[j] of band b
};

PANO_HD Walker walk_start(const uint32_t* gs, const uint16_t* st, const int* lo, const int* hi, const int* zs, int w,
                          int nb, int a, int x) {
    int l = 0, r = nb - 1;  // largest b with zs[b] <= x (zs[first kept band] = -1)
    while (l < r) {
        const int m = (l + r + 1) >> 1;
        if (PANO_AT(zs, m, nb, 534) <= x) l = m;
        else r = m - 1;
    }
    Walker k;
    k.b = l;
    k.j = PANO_AT(lo, l, nb, 535);
    for (int it = 0; it < w && k.j + 1 < PANO_AT(hi, l, nb, 535); ++it) {
        const int p = PANO_AT(st, k.j, w, 536), q = PANO_AT(st, k.j + 1, w, 536);
        if (!owns(f_of(gs, w, a, p), p, f_of(gs, w, a, q), q, x)) break;
        ++k.j;
    }
    return k;
}

// moves the walker to the owner of column x (x not left of the last one)
// and returns d2(x)
PANO_HD long long walk_to(const uint32_t* gs, const uint16_t* st, const int* lo, const int* hi, const int* nxt, int w,
                          int nb, int a, int x, Walker* k) {
    for (int it = 0; it < w; ++it) {
        int b = k->b, j = k->j + 1;
        if (j >= PANO_AT(hi, b, nb, 537)) {
            if (b + 1 >= nb) break;
            b = PANO_AT(nxt, b + 1, nb, 538);
            if (b >= nb) break;
            j = lo[b];
        }
        const int p = PANO_AT(st, k->j, w, 539), q = PANO_AT(st, j, w, 539);
        if (!owns(f_of(gs, w, a, p), p, f_of(gs, w, a, q), q, x)) break;
        k->b = b;
        k->j = j;
    }
    const int s = PANO_AT(st, k->j, w, 540);
    const long long dx = x - s;
    return dx * dx + f_of(gs, w, a, s);
}

}  // namespace edt
}  // namespace pano
