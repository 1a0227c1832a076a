// Host-side index tables of a dielectric G-sphere on an n0 x n1 x n2 grid, the maps the pair
// kernels follow to prune the forward transform of a pair product down to the sphere's points:
//   kz       the kept last-axis frequencies (the z indices, mod n2, of the sphere's points),
//   pack[i]  point i as k0 | k1 << 8 | (position of its k2 in kz) << 16,
//   cells    the (kz position, k1) cells that hold points, ordered by (kz position, k1), each
//            as kz position << 8 | k1, with the points of cell d at cg[cstart[d] .. cstart[d+1]),
//   cpts[m]  (point index, k0 | cell << 8) in that cell order.
// Plain C++ (no CUDA): the library builds its device tables from it, and the CPU tests check that
// every index the kernels derive from it stays inside its buffer.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <utility>
#include <vector>

namespace gw {

struct SpherePlanHost {
    int K2 = 0, K12 = 0;
    std::vector<int> kz;
    std::vector<int32_t> pack;
    std::vector<int> cstart, cg;
    std::vector<int32_t> cell;
    std::vector<std::pair<int, int>> cpts;
};

inline int plan_mod(int a, int n) { return ((a % n) + n) % n; }

// g: [ng][3] Miller indices with every component inside (-n/2, n/2) (the caller checks).
inline void build_sphere_plan(const int n[3], int ng, const int32_t *g, SpherePlanHost &p)
{
    std::vector<int> present(n[2], 0), pos(n[2], -1);
    for (int i = 0; i < ng; ++i) present[plan_mod(g[3 * i + 2], n[2])] = 1;
    p.kz.clear();
    for (int k = 0; k < n[2]; ++k)
        if (present[k]) {
            pos[k] = (int)p.kz.size();
            p.kz.push_back(k);
        }
    p.K2 = (int)p.kz.size();
    p.pack.assign(ng, 0);
    for (int i = 0; i < ng; ++i) {
        const int k0 = plan_mod(g[3 * i], n[0]), k1 = plan_mod(g[3 * i + 1], n[1]);
        const int k2 = pos[plan_mod(g[3 * i + 2], n[2])];
        p.pack[i] = k0 | (k1 << 8) | (k2 << 16);
    }
    // group the points by their (kz position, k1) cell
    std::vector<std::pair<int, int>> key(ng);
    for (int i = 0; i < ng; ++i) key[i] = {(p.pack[i] >> 16) * n[1] + ((p.pack[i] >> 8) & 255), i};
    std::sort(key.begin(), key.end());
    p.cg.assign(ng, 0);
    p.cstart.clear();
    for (int i = 0; i < ng; ++i) {
        if (i == 0 || key[i].first != key[i - 1].first) p.cstart.push_back(i);
        p.cg[i] = key[i].second;
    }
    p.cstart.push_back(ng);
    p.K12 = (int)p.cstart.size() - 1;
    p.cell.assign(p.K12, 0);
    p.cpts.assign(ng, {0, 0});
    for (int d = 0; d < p.K12; ++d) {
        const int i = p.cg[p.cstart[d]];
        p.cell[d] = (p.pack[i] >> 16) << 8 | ((p.pack[i] >> 8) & 255);
        for (int m = p.cstart[d]; m < p.cstart[d + 1]; ++m) p.cpts[m] = {p.cg[m], (p.pack[p.cg[m]] & 255) | d << 8};
    }
}

} // namespace gw
