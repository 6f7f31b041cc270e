// Host run of the row pass of the Eq. (1) distance transform: the steps of
// edt_row.cuh (compiled here by a host compiler, with an index check that
// counts every access outside its array) in the order edt_row_kernel runs
// them, thread by thread and round by round, on random rows; every d2 is
// compared with a brute-force minimum over all sites. Prints
// "rows R bad B oob O"; exits non-zero on any mismatch or bad index.
// Usage: edt_row_host [trials]
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>
#include <random>
#include <algorithm>
#include <climits>
static long long g_oob = 0;
template <class T> T& at(T* b, long long off, long long n, int site) {
    if (off < 0 || off >= n) { if (!g_oob) fprintf(stderr, "OOB site %d off %lld n %lld\n", site, off, n); ++g_oob; off = off < 0 ? 0 : n - 1; }
    return b[off];
}
#define PANO_AT(base, off, n, site) (at((base), (long long)(off), (long long)(n), (site)))
#include "edt_row.cuh"
using namespace pano::edt;

// d2 of one area's row by the emulated kernel (NB threads)
static bool row_pass1(const std::vector<uint16_t>& gsv, int w, int NB, std::vector<long long>& d2, bool* any) {
    std::vector<uint16_t> gs = gsv, st(w);
    std::vector<int> lo(NB), hi(NB), gf(NB), gl(NB), zs(NB);
    const int bw = (w + NB - 1) / NB;
    {
        std::vector<int> ls(NB), fe(NB), ps(NB), sf(NB);
        for (int t = 0; t < NB; ++t) { const int x0 = std::min(w, t * bw), x1 = std::min(w, x0 + bw); band_run_edges(gs.data(), w, x0, x1, &ls[t], &fe[t]); }
        int m = INT_MIN; for (int t = 0; t < NB; ++t) { m = std::max(m, ls[t]); ps[t] = m; }
        m = INT_MAX; for (int t = NB - 1; t >= 0; --t) { m = std::min(m, fe[t]); sf[t] = m; }
        for (int t = 0; t < NB; ++t) {
            const int x0 = std::min(w, t * bw), x1 = std::min(w, x0 + bw);
            int L = -1, R = w;
            if (x0 < x1) {
                const int u = (x0 == 0 || gs[x0] != gs[x0 - 1]) ? x0 : (t > 0 ? ps[t - 1] : 0);
                const int v = (x1 == w || gs[x1 - 1] != gs[x1]) ? x1 - 1 : (t + 1 < NB ? sf[t + 1] : w - 1);
                L = u - 1; R = v + 1;
            }
            edge_runs_hidden(gs.data(), st.data(), w, x0, x1, L, R);
        }
        for (int q = 0; q < w; ++q) if (st[q]) gs[q] = (uint16_t)kNoSite;
    }
    for (int t = 0; t < NB; ++t) {
        const int x0 = std::min(w, t * bw), x1 = std::min(w, x0 + bw);
        int k = band_envelope(gs.data(), st.data(), w, x0, x1);
        lo[t] = x0; hi[t] = x0 + k; gf[t] = k ? t : -1; gl[t] = k ? t : -1;
    }
    bool ok = true;
    for (int s = 1; s < NB; s <<= 1)
        for (int lg = 0; lg < NB; ++lg)
            if ((lg & (2 * s - 1)) == 0 && lg + s < NB) {
                int lf = gf[lg], ll = gl[lg], rf = gf[lg + s], rl = gl[lg + s];
                if (rf >= 0) {
                    if (lf < 0) gf[lg] = rf;
                    else if (!merge_groups(gs.data(), st.data(), lo.data(), hi.data(), w, NB, lf, ll, rf, rl)) ok = false;
                    gl[lg] = rl;
                }
            }
    *any = gf[0] >= 0;
    int pv = -1;
    for (int b = 0; b < NB; ++b) { if (hi[b] > lo[b]) pv = b; gf[b] = pv; }
    int nx = NB;
    for (int b = NB - 1; b >= 0; --b) { if (hi[b] > lo[b]) nx = b; gl[b] = nx; }
    for (int b = 0; b < NB; ++b)
        if (hi[b] > lo[b]) {
            const int pb = b > 0 ? gf[b - 1] : -1; int z = -1;
            if (pb >= 0) { int p = st[hi[pb]-1], q = st[lo[b]]; z = region_start(f_of(gs.data(), w, p), p, f_of(gs.data(), w, q), q, w); }
            zs[b] = z;
        }
    for (int b = 0; b < NB; ++b) if (hi[b] <= lo[b]) { int n = gl[b]; zs[b] = n < NB ? zs[n] : w; }
    d2.assign(w, -1);
    for (int t = 0; t < NB; ++t) {
        const int x0 = std::min(w, t * bw), x1 = std::min(w, x0 + bw);
        if (x0 >= x1 || !*any) continue;
        Walker k = walk_start(gs.data(), st.data(), lo.data(), hi.data(), zs.data(), w, NB, x0);
        for (int x = x0; x < x1; ++x) {
            if ((x * 7 + t) % 3 == 0 && x != x0) continue;  // lazy walk: skip some columns
            d2[x] = walk_to(gs.data(), st.data(), lo.data(), hi.data(), gl.data(), w, NB, x, &k);
        }
    }
    return ok;
}

static bool row_pass(const std::vector<uint32_t>& g, int w, int NB, std::vector<long long> d2[2], bool any[2]) {
    bool ok = true;
    for (int a = 0; a < 2; ++a) {
        std::vector<uint16_t> ga(w);
        for (int x = 0; x < w; ++x) ga[x] = (uint16_t)((g[x] >> (16 * a)) & 0xFFFF);
        ok &= row_pass1(ga, w, NB, d2[a], &any[a]);
    }
    return ok;
}

int main(int argc, char** argv) {
    const int trials = argc > 1 ? atoi(argv[1]) : 6000;
    std::mt19937_64 rng(1234);
    long long rows = 0, bad = 0;
    const int NBs[] = {2, 4, 8, 16, 64, 256};
    for (int trial = 0; trial < trials; ++trial) {
        int w = 1 + (int)(rng() % (trial < trials / 2 ? 80 : 3000));
        int NB = NBs[rng() % 6];
        std::vector<uint32_t> g(w);
        int mode = rng() % 7;
        const int S = 1 + (int)(rng() % 60), D = 1 + (int)(rng() % 90);
        for (int x = 0; x < w; ++x) {
            uint32_t gv[2];
            for (int a = 0; a < 2; ++a) {
                uint32_t v;
                switch (mode) {
                    case 0: v = (rng() % 4 == 0) ? kNoSite : (uint32_t)(rng() % 50); break;
                    case 1: v = (rng() % 20 == 0) ? (uint32_t)(rng() % 3000) : kNoSite; break;   // sparse
                    case 2: v = (uint32_t)(rng() % 65535); break;                                  // huge
                    case 3: v = (x < w / 3 && a == 0) || (x > 2 * w / 3 && a == 1) ? 0 : (rng() % 3 ? kNoSite : (uint32_t)(rng() % 200)); break;
                    case 4: v = (uint32_t)(rng() % 3); break;                                      // many ties
                    case 6: v = (uint32_t)((((x + 13 * a) / S) * D + (x / (7 * S)) % 3 * 5) % 2000); break;   // staircases
                    default: v = (rng() % 2) ? kNoSite : (uint32_t)((x * 37 + a * 11) % 17); break;
                }
                gv[a] = v;
            }
            g[x] = gv[0] | (gv[1] << 16);
        }
        std::vector<long long> d2[2]; bool any[2];
        bool ok = row_pass(g, w, NB, d2, any);
        if (!ok) { ++bad; fprintf(stderr, "limit reached trial %d\n", trial); }
        for (int a = 0; a < 2; ++a) {
            bool has = false;
            for (int x = 0; x < w; ++x) if (((g[x] >> (16*a)) & 0xFFFF) != kNoSite) has = true;
            if (has != any[a]) { ++bad; fprintf(stderr, "any mismatch trial %d\n", trial); }
            if (!has) continue;
            for (int x = 0; x < w; ++x) {
                if (d2[a][x] < 0) continue;
                long long best = LLONG_MAX;
                for (int q = 0; q < w; ++q) {
                    uint32_t v = (g[q] >> (16*a)) & 0xFFFF; if (v == kNoSite) continue;
                    long long d = (long long)(x - q) * (x - q) + (long long)v * v; best = std::min(best, d);
                }
                if (best != d2[a][x]) { if (bad < 10) fprintf(stderr, "trial %d w %d NB %d mode %d a %d x %d got %lld want %lld\n", trial, w, NB, mode, a, x, d2[a][x], best); ++bad; }
            }
        }
        ++rows;
    }
    printf("rows %lld bad %lld oob %lld\n", rows, bad, g_oob);
    return bad || g_oob;
}
