// Host-side check of the library's mesh ordering and tiling (compiled by tests/test_mesh_cpu.py).
// Builds a jittered square mesh and prints "ok" lines or the first violated property.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <set>
#include <vector>

#include "internal.h"

using namespace festung;

static int fail(const char *m) {
    std::printf("FAIL %s\n", m);
    return 1;
}

int main(int argc, char **argv) {
    const int n = argc > 1 ? std::atoi(argv[1]) : 13;
    const int TE = argc > 2 ? std::atoi(argv[2]) : 64;
    std::vector<double> cV;
    std::vector<int32_t> V0T;
    srand(7);
    for (int ix = 0; ix <= n; ++ix)
        for (int iy = 0; iy <= n; ++iy) {
            double x = ix * 1.0 / n, y = iy * 1.0 / n;
            if (ix > 0 && ix < n && iy > 0 && iy < n) {
                x += 0.2 / n * (2.0 * rand() / RAND_MAX - 1.0);
                y += 0.2 / n * (2.0 * rand() / RAND_MAX - 1.0);
            }
            cV.push_back(x);
            cV.push_back(y);
        }
    auto vid = [&](int ix, int iy) { return iy + ix * (n + 1); };
    for (int ix = 0; ix < n; ++ix)
        for (int iy = 0; iy < n; ++iy) {
            V0T.insert(V0T.end(), {vid(ix, iy), vid(ix + 1, iy), vid(ix, iy + 1)});
        }
    for (int ix = 0; ix < n; ++ix)
        for (int iy = 0; iy < n; ++iy) {
            V0T.insert(V0T.end(), {vid(ix + 1, iy), vid(ix + 1, iy + 1), vid(ix, iy + 1)});
        }
    const int64_t K = V0T.size() / 3;
    std::vector<int8_t> bdr(3 * K, 0);
    for (int64_t k = 0; k < K; ++k)
        for (int e = 0; e < 3; ++e) {
            const int a = V0T[3 * k + (e + 1) % 3], b = V0T[3 * k + (e + 2) % 3];
            const int ax = a / (n + 1), ay = a % (n + 1), bx = b / (n + 1), by = b % (n + 1);
            if ((ax == 0 && bx == 0) || (ax == n && bx == n)) bdr[3 * k + e] = 1;  // Dirichlet x = 0, 1
            if ((ay == 0 && by == 0) || (ay == n && by == n)) bdr[3 * k + e] = 2;  // Neumann y = 0, 1
        }
    std::vector<double> B;
    std::vector<int32_t> nbr;
    std::string err;
    if (build_mesh(cV.data(), cV.size() / 2, V0T.data(), K, bdr.data(), B, nbr, err)) return fail(err.c_str());
    MeshOrder o;
    order_and_tile(cV.data(), V0T.data(), K, B, nbr, TE, o);
    // permutation
    std::vector<int> seen(K, 0);
    for (int64_t i = 0; i < K; ++i) {
        if (o.perm[i] < 0 || o.perm[i] >= K || seen[o.perm[i]]++) return fail("perm is not a permutation");
        if (o.inv[o.perm[i]] != i) return fail("inv is not the inverse");
    }
    std::printf("ok perm\n");
    // geometry and neighbours in internal order
    for (int64_t i = 0; i < K; ++i) {
        const int64_t u = o.perm[i];
        for (int c = 0; c < 4; ++c)
            if (o.B[c * K + i] != B[c * K + u]) return fail("B not permuted");
        for (int e = 0; e < 3; ++e) {
            const int32_t code = o.nbr[e * K + i];
            if (code < 0) {
                if (code != nbr[e * K + u]) return fail("boundary code changed");
                continue;
            }
            const int64_t k2 = code >> 2;
            const int n2 = code & 3;
            if (o.nbr[n2 * K + k2] != (int32_t)((i << 2) | e)) return fail("neighbour relation not symmetric");
            if (o.perm[k2] != (nbr[e * K + u] >> 2)) return fail("neighbour not remapped");
        }
    }
    std::printf("ok neighbours\n");
    // tiles, halos, slots
    const int64_t T = (K + TE - 1) / TE;
    if ((int64_t)o.halo_ptr.size() != T + 1) return fail("halo_ptr size");
    for (int64_t t = 0; t < T; ++t) {
        const int64_t s0 = t * TE, s1 = std::min<int64_t>(K, s0 + TE);
        std::set<int32_t> hs;
        for (int h = o.halo_ptr[t]; h < o.halo_ptr[t + 1]; ++h) {
            const int32_t e = o.halo[h];
            if (e >= s0 && e < s1) return fail("halo element inside its tile");
            if (!hs.insert(e).second) return fail("halo element repeated");
            for (int n2 = 0; n2 < 3; ++n2) {
                const int32_t code = o.nbr[n2 * K + e], sl = o.halo_slot[3 * h + n2];
                if (code < 0) {
                    if (sl != -1) return fail("halo boundary slot");
                    continue;
                }
                const int64_t k2 = code >> 2;
                if (sl == -2) {
                    if ((k2 >= s0 && k2 < s1) || hs.count((int32_t)k2)) {
                        // k2 may appear later in the halo list; check against the full list
                        bool in = false;
                        for (int q = o.halo_ptr[t]; q < o.halo_ptr[t + 1]; ++q) in |= o.halo[q] == k2;
                        if ((k2 >= s0 && k2 < s1) || in) return fail("resident neighbour marked non-resident");
                    }
                } else {
                    const int64_t want = sl < TE ? s0 + sl : o.halo[o.halo_ptr[t] + sl - TE];
                    if (want != k2) return fail("halo neighbour slot wrong");
                }
            }
        }
        for (int64_t i = s0; i < s1; ++i)
            for (int e = 0; e < 3; ++e) {
                const int32_t code = o.nbr[e * K + i], sl = o.slot[e * K + i];
                if (code < 0) {
                    if (sl != -1) return fail("boundary slot");
                    continue;
                }
                const int64_t k2 = code >> 2;
                const int64_t want = sl < TE ? s0 + sl : o.halo[o.halo_ptr[t] + sl - TE];
                if (sl < 0 || want != k2) return fail("tile slot wrong");
            }
    }
    std::printf("ok tiles %ld max_halo %d\n", (long)T, o.max_halo);
    // Dirichlet-lift flags
    for (int64_t i = 0; i < K; ++i) {
        bool own = false, near = false;
        for (int e = 0; e < 3; ++e) {
            const int32_t code = o.nbr[e * K + i];
            if (code == -1) own = true;
            if (code >= 0)
                for (int f = 0; f < 3; ++f) near |= o.nbr[f * K + (code >> 2)] == -1;
        }
        if (((o.lift[i] & 1) != 0) != own || ((o.lift[i] & 2) != 0) != (own || near)) return fail("lift flags");
    }
    std::printf("ok lift\n");
    // tile sizes: whole warps, at most 256, and the tiles fill whole waves of resident blocks
    for (int64_t KK : {1L, 31L, 72L, 8192L, 131072L, 131073L, 2097152L})
        for (int R : {1, 152, 304, 456}) {
            const int sms = R < 152 ? R : 152;
            const int te = tile_size(KK, R, sms);
            if (te < 32 || te > 256 || te % 32) return fail("tile size range");
            if ((KK + 255) / 256 <= sms) {
                if (te != 256) return fail("tiles split although SMs are idle");
                continue;
            }
            const int64_t waves = (KK + 256L * R - 1) / (256L * R);
            const int64_t tiles = (KK + te - 1) / te;
            if (te > 32 && tiles > waves * R) return fail("tiles exceed whole waves");
            if (te - 32 >= (KK + waves * R - 1) / (waves * R)) return fail("tile size larger than needed");
        }
    std::printf("ok tile_size\n");
    return 0;
}
