// Host check of the index maps the pair kernels follow (built and run by tests/test_plans.py on
// the CPU).  Reads "n0 n1 n2 ng" and then ng Miller triples; builds the sphere's tables with the
// library's own builder (csrc/sphere_plan.h) and walks every index the kernels derive from them
// and from the radix plans of the grid (csrc/fft_tf.cuh), checking each against the extent of the
// buffer it addresses.  Prints "OK" or the first violations; exits non-zero on a violation.
#include <cstdio>
#include <string>
#include <vector>

#include "../../paper_2509_23018_gb300/csrc/fft_tf.cuh"
#include "../../paper_2509_23018_gb300/csrc/sphere_plan.h"

static int fails = 0;
#define REQUIRE(c, ...)                                                                                \
    do {                                                                                               \
        if (!(c)) {                                                                                    \
            if (fails++ < 5) {                                                                         \
                std::printf("FAIL %s:%d: ", __FILE__, __LINE__);                                       \
                std::printf(__VA_ARGS__);                                                              \
                std::printf("\n");                                                                     \
            }                                                                                          \
        }                                                                                              \
    } while (0)

// Every Stockham stage of a plan: inputs, twiddles and outputs inside the line, the outputs a
// permutation (each index written once); the pruned last stage's reads for every output k.
static void check_plan(int n, const gw::RadPlan &p, bool pruned)
{
    int prod = 1;
    for (int s = 0; s < p.nst; ++s) prod *= p.r[s];
    REQUIRE(prod == n, "plan of %d multiplies to %d", n, prod);
    const int full = pruned ? p.nst - 1 : p.nst;
    int ns = 1;
    for (int s = 0; s < full; ++s) {
        const int R = p.r[s], nb = n / R, tstride = n / (ns * R);
        std::vector<int> written(n, 0);
        for (int j = 0; j < nb; ++j) {
            const int kk = j % ns;
            for (int r = 0; r < R; ++r) {
                REQUIRE(j + r * nb < n, "n %d stage %d input %d", n, s, j + r * nb);
                REQUIRE(r * kk * tstride < n, "n %d stage %d twiddle %d", n, s, r * kk * tstride);
                const int o = (j / ns) * (ns * R) + kk + r * ns;
                REQUIRE(o >= 0 && o < n, "n %d stage %d output %d", n, s, o);
                if (o >= 0 && o < n) ++written[o];
            }
        }
        for (int i = 0; i < n; ++i) REQUIRE(written[i] == 1, "n %d stage %d output %d written %d times", n, s, i, written[i]);
        ns *= R;
    }
    if (pruned) {
        const int R = p.r[p.nst - 1], NS = n / R;
        REQUIRE(NS == ns, "n %d pruned stage spacing %d vs %d", n, NS, ns);
        for (int k = 0; k < n; ++k) {
            const int j = k % NS;
            int e = 0;
            for (int r = 0; r < R; ++r) {
                REQUIRE(j + r * NS < n, "n %d pruned output %d reads %d", n, k, j + r * NS);
                if (r) {
                    e += k;
                    if (e >= n) e -= n;
                    REQUIRE(e >= 0 && e < n, "n %d pruned output %d twiddle %d", n, k, e);
                }
            }
        }
    }
}

int main(int argc, char **argv)
{
    // --corrupt: swap two cells of the built tables (the checker's own test)
    const bool corrupt = argc > 1 && std::string(argv[1]) == "--corrupt";
    int n[3], ng;
    if (std::scanf("%d %d %d %d", &n[0], &n[1], &n[2], &ng) != 4) return 2;
    std::vector<int32_t> g(3 * (size_t)ng);
    for (int i = 0; i < 3 * ng; ++i)
        if (std::scanf("%d", &g[i]) != 1) return 2;
    for (int a = 0; a < 3; ++a) {
        check_plan(n[a], gw::make_rad_plan(n[a]), false);
        if (n[a] % 2 == 0 || n[a] % 3 == 0 || n[a] % 5 == 0) check_plan(n[a], gw::make_prune_plan(n[a]), true);
    }
    gw::SpherePlanHost p;
    gw::build_sphere_plan(n, ng, g.data(), p);
    if (corrupt && p.K12 > 1) std::swap(p.cell[0], p.cell[p.K12 - 1]);

    // kept last-axis frequencies: increasing, inside the axis; every point's position valid
    REQUIRE(p.K2 >= 1 && p.K2 == (int)p.kz.size(), "K2 %d", p.K2);
    for (int q = 0; q < p.K2; ++q) {
        REQUIRE(p.kz[q] >= 0 && p.kz[q] < n[2], "kz[%d] = %d", q, p.kz[q]);
        if (q) REQUIRE(p.kz[q] > p.kz[q - 1], "kz not increasing at %d", q);
    }
    for (int i = 0; i < ng; ++i) {
        const int k0 = p.pack[i] & 255, k1 = (p.pack[i] >> 8) & 255, q = p.pack[i] >> 16;
        REQUIRE(k0 < n[0] && k1 < n[1] && q < p.K2, "pack[%d] = %d %d %d", i, k0, k1, q);
        // the point's own frequency: (g mod n) on every axis
        REQUIRE(k0 == gw::plan_mod(g[3 * i], n[0]) && k1 == gw::plan_mod(g[3 * i + 1], n[1]) &&
                    p.kz[q] == gw::plan_mod(g[3 * i + 2], n[2]),
                "pack[%d] does not address G %d %d %d", i, g[3 * i], g[3 * i + 1], g[3 * i + 2]);
    }
    // cells: sorted by (kz position, k1) (the kernels' per-column ranges rely on it), the points
    // of cell d in cstart[d] .. cstart[d + 1], every point once
    REQUIRE(p.K12 >= 1 && (int)p.cstart.size() == p.K12 + 1 && p.cstart[0] == 0 && p.cstart[p.K12] == ng, "cstart");
    std::vector<int> seen(ng, 0);
    for (int d = 0; d < p.K12; ++d) {
        const int q = p.cell[d] >> 8, k1 = p.cell[d] & 255;
        REQUIRE(q < p.K2 && k1 < n[1], "cell[%d] = %d %d", d, q, k1);
        if (d) REQUIRE(p.cell[d] > p.cell[d - 1], "cells not increasing at %d", d);
        REQUIRE(p.cstart[d] < p.cstart[d + 1], "empty cell %d", d);
        for (int m = p.cstart[d]; m < p.cstart[d + 1]; ++m) {
            const int pt = p.cpts[m].first, k0 = p.cpts[m].second & 255, dd = p.cpts[m].second >> 8;
            REQUIRE(pt >= 0 && pt < ng, "cpts[%d] point %d", m, pt);
            if (pt < 0 || pt >= ng) continue;
            ++seen[pt];
            REQUIRE(dd == d && k0 < n[0], "cpts[%d] cell %d k0 %d", m, dd, k0);
            REQUIRE(((p.pack[pt] >> 16) << 8 | ((p.pack[pt] >> 8) & 255)) == p.cell[d], "point %d not in cell %d", pt, d);
        }
    }
    for (int i = 0; i < ng; ++i) REQUIRE(seen[i] == 1, "point %d listed %d times", i, seen[i]);

    // the pair kernels' uses of the tables (cubic grids: one line length N for every axis)
    if (n[0] == n[1] && n[1] == n[2]) {
        const int N = n[0], CS = N + 1;
        // i1 cells read column q = cell >> 8 of the C buffer [K2][CS] at k1 < N
        for (int d = 0; d < p.K12; ++d) REQUIRE((p.cell[d] >> 8) * CS + (p.cell[d] & 255) < p.K2 * CS, "cell %d", d);
        // phase 2 in batches of NB cell columns: a point's column inside its batch
        for (int NB : {15, 23, 31, 45}) {
            for (int d0 = 0; d0 < p.K12; d0 += NB) {
                const int nbat = std::min(NB, p.K12 - d0);
                for (int m = p.cstart[d0]; m < p.cstart[d0 + nbat]; ++m) {
                    const int c = (p.cpts[m].second >> 8) - d0;
                    REQUIRE(c >= 0 && c < nbat, "batch %d point %d column %d", d0, m, c);
                }
            }
        }
        // the middle/first-axis kernel of the tensor-core route: per slab pair, column col =
        // sl K2 + q; the cells of kept column q form the range [first cell with q' >= q, ...)
        std::vector<int> cofs(p.K2 + 1);
        for (int q = 0; q <= p.K2; ++q) {
            int lo = 0, hi = p.K12;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((p.cell[mid] >> 8) < q) lo = mid + 1;
                else hi = mid;
            }
            cofs[q] = lo;
        }
        REQUIRE(cofs[0] == 0 && cofs[p.K2] == p.K12, "column ranges do not cover the cells");
        for (int q = 0; q < p.K2; ++q)
            for (int d = cofs[q]; d < cofs[q + 1]; ++d) REQUIRE((p.cell[d] >> 8) == q, "cell %d outside column %d", d, q);
        // the tensor-core product: 2 K2 real columns per conduction band inside a 64-column tile
        if (N == 48 && p.K2 <= 16) {
            const int ct = std::min(4, 64 / (2 * p.K2));
            REQUIRE(ct >= 1 && ct * 2 * p.K2 <= 64, "conduction bands per tile %d", ct);
        }
    }
    if (fails) {
        std::printf("%d violations\n", fails);
        return 1;
    }
    std::printf("OK K2 %d K12 %d\n", p.K2, p.K12);
    return 0;
}
