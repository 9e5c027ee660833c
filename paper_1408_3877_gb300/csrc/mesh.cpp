// Grid lists (Sec. 3.1, Tab. 1): neighbour relation through shared edges, the affine
// maps B_k of eq. affinemappings, and validation of the input mesh.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace festung {

int build_mesh(const double *coordV, int64_t numV, const int32_t *V0T, int64_t K,
               const int8_t *bdr, std::vector<double> &B, std::vector<int32_t> &nbr,
               std::string &err) {
    if (K >= (int64_t(1) << 29)) {
        err = "too many triangles (limit 2^29 - 1)";
        return FESTUNG_EINVAL;
    }
    for (int64_t v = 0; v < 2 * numV; ++v)
        if (!std::isfinite(coordV[v])) {
            err = "non-finite vertex coordinate";
            return FESTUNG_EDATA;
        }
    for (int64_t i = 0; i < 3 * K; ++i) {
        if (V0T[i] < 0 || V0T[i] >= numV) {
            err = "vertex index out of range in V0T";
            return FESTUNG_EMESH;
        }
        if (bdr[i] < 0 || bdr[i] > 2) {
            err = "boundary type must be 0, 1 or 2";
            return FESTUNG_EMESH;
        }
    }
    B.assign(4 * K, 0.0);
    for (int64_t k = 0; k < K; ++k) {
        const double *a1 = coordV + 2 * int64_t(V0T[3 * k + 0]);
        const double *a2 = coordV + 2 * int64_t(V0T[3 * k + 1]);
        const double *a3 = coordV + 2 * int64_t(V0T[3 * k + 2]);
        const double b11 = a2[0] - a1[0], b12 = a3[0] - a1[0];
        const double b21 = a2[1] - a1[1], b22 = a3[1] - a1[1];
        const double det = b11 * b22 - b12 * b21;
        if (!(det > 0.0)) {
            err = "triangle " + std::to_string(k) + " is clockwise or degenerate (det B <= 0)";
            return FESTUNG_EMESH;
        }
        B[0 * K + k] = b11;
        B[1 * K + k] = b12;
        B[2 * K + k] = b21;
        B[3 * K + k] = b22;
    }
    // half-edges (k, n): from vertex n+1 to n+2; key = (min, max) vertex pair
    std::vector<int64_t> key(3 * K);
    std::vector<int64_t> idx(3 * K);
    for (int64_t k = 0; k < K; ++k)
        for (int n = 0; n < 3; ++n) {
            const int64_t va = V0T[3 * k + (n + 1) % 3], vb = V0T[3 * k + (n + 2) % 3];
            if (va == vb) {
                err = "triangle with a repeated vertex";
                return FESTUNG_EMESH;
            }
            key[3 * k + n] = std::min(va, vb) * numV + std::max(va, vb);
            idx[3 * k + n] = 3 * k + n;
        }
    std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
        return key[a] < key[b] || (key[a] == key[b] && a < b);
    });
    nbr.assign(3 * K, 0);
    int64_t i = 0;
    while (i < 3 * K) {
        int64_t j = i + 1;
        while (j < 3 * K && key[idx[j]] == key[idx[i]]) ++j;
        const int64_t cnt = j - i;
        if (cnt > 2) {
            err = "edge shared by more than two triangles";
            return FESTUNG_EMESH;
        }
        const int64_t h0 = idx[i];
        const int64_t k0 = h0 / 3;
        const int n0 = int(h0 % 3);
        if (cnt == 1) {
            const int t = bdr[h0];
            if (t == FESTUNG_BDR_INTERIOR) {
                err = "boundary edge of triangle " + std::to_string(k0) + " has no boundary type";
                return FESTUNG_EMESH;
            }
            nbr[n0 * K + k0] = (t == FESTUNG_BDR_DIRICHLET) ? -1 : -2;
        } else {
            const int64_t h1 = idx[i + 1];
            const int64_t k1 = h1 / 3;
            const int n1 = int(h1 % 3);
            if (bdr[h0] != 0 || bdr[h1] != 0) {
                err = "interior edge marked as boundary";
                return FESTUNG_EMESH;
            }
            // consistent counter-clockwise orientation: the shared edge runs oppositely
            const int64_t a0 = V0T[3 * k0 + (n0 + 1) % 3], a1v = V0T[3 * k1 + (n1 + 1) % 3];
            if (a0 == a1v) {
                err = "neighbouring triangles traverse their shared edge in the same direction";
                return FESTUNG_EMESH;
            }
            nbr[n0 * K + k0] = int32_t((k1 << 2) | n1);
            nbr[n1 * K + k1] = int32_t((k0 << 2) | n0);
        }
        i = j;
    }
    return FESTUNG_OK;
}

}  // namespace festung

namespace festung {

namespace {

// spread the low 21 bits of v to the even bit positions (one axis of a 2-D Morton key)
uint64_t spread2(uint64_t v) {
    v &= 0x1fffffULL;
    v = (v | (v << 16)) & 0x0000ffff0000ffffULL;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffULL;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0fULL;
    v = (v | (v << 2)) & 0x3333333333333333ULL;
    v = (v | (v << 1)) & 0x5555555555555555ULL;
    return v;
}

}  // namespace

void order_mesh(const double *coordV, const int32_t *V0T, int64_t K, const std::vector<double> &B_usr,
                const std::vector<int32_t> &nbr_usr, MeshOrder &o) {
    // Morton order of the triangle centroids: nearby triangles get nearby indices, so a
    // tile of TE consecutive triangles is a compact patch with a short boundary.
    std::vector<double> cx(K), cy(K);
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int64_t k = 0; k < K; ++k) {
        double sx = 0, sy = 0;
        for (int v = 0; v < 3; ++v) {
            sx += coordV[2 * int64_t(V0T[3 * k + v])];
            sy += coordV[2 * int64_t(V0T[3 * k + v]) + 1];
        }
        cx[k] = sx / 3.0;
        cy[k] = sy / 3.0;
        x0 = std::min(x0, cx[k]);
        x1 = std::max(x1, cx[k]);
        y0 = std::min(y0, cy[k]);
        y1 = std::max(y1, cy[k]);
    }
    const double span = std::max(std::max(x1 - x0, y1 - y0), 1e-300);
    const double scale = double((1 << 21) - 1) / span;
    std::vector<uint64_t> key(K);
    for (int64_t k = 0; k < K; ++k) {
        const uint64_t qx = (uint64_t)((cx[k] - x0) * scale), qy = (uint64_t)((cy[k] - y0) * scale);
        key[k] = spread2(qx) | (spread2(qy) << 1);
    }
    o.perm.resize(K);
    for (int64_t k = 0; k < K; ++k) o.perm[k] = (int32_t)k;
    std::stable_sort(o.perm.begin(), o.perm.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    o.inv.assign(K, 0);
    for (int64_t i = 0; i < K; ++i) o.inv[o.perm[i]] = (int32_t)i;
    // geometry and neighbour codes in internal order
    o.B.assign(4 * K, 0.0);
    o.nbr.assign(3 * K, 0);
    for (int64_t i = 0; i < K; ++i) {
        const int64_t u = o.perm[i];
        for (int c = 0; c < 4; ++c) o.B[c * K + i] = B_usr[c * K + u];
        for (int n = 0; n < 3; ++n) {
            const int32_t code = nbr_usr[n * K + u];
            o.nbr[n * K + i] = code >= 0 ? (int32_t)((int64_t(o.inv[code >> 2]) << 2) | (code & 3)) : code;
        }
    }
    lift_flags(o.nbr, K, o.lift);
}

void lift_flags(const std::vector<int32_t> &nbr, int64_t K, std::vector<uint8_t> &lift) {
    // triangles whose right-hand side sees the Dirichlet lift: bit 0 = has a Dirichlet
    // edge, bit 1 = it or an interior neighbour has one
    lift.assign(K, 0);
    for (int64_t i = 0; i < K; ++i)
        for (int n = 0; n < 3; ++n)
            if (nbr[n * K + i] == -1) lift[i] |= 3;
    for (int64_t i = 0; i < K; ++i)
        for (int n = 0; n < 3; ++n) {
            const int32_t code = nbr[n * K + i];
            if (code >= 0 && (lift[code >> 2] & 1)) lift[i] |= 2;
        }
}

void tile_mesh(const std::vector<int32_t> &nbr, int64_t K, int TE, MeshOrder &o) {
    // tiles of TE consecutive triangles; halo = interior neighbours outside the tile
    o.TE = TE;
    const int64_t T = (K + TE - 1) / TE;
    o.halo_ptr.assign(T + 1, 0);
    o.halo.clear();
    o.halo_slot.clear();
    o.slot.assign(3 * K, -1);
    o.max_halo = 0;
    std::vector<int32_t> h;
    for (int64_t t = 0; t < T; ++t) {
        const int64_t s0 = t * TE, s1 = std::min(K, s0 + TE);
        h.clear();
        for (int64_t i = s0; i < s1; ++i)
            for (int n = 0; n < 3; ++n) {
                const int32_t code = nbr[n * K + i];
                if (code < 0) continue;
                const int64_t k2 = code >> 2;
                if (k2 < s0 || k2 >= s1) h.push_back((int32_t)k2);
            }
        std::sort(h.begin(), h.end());
        h.erase(std::unique(h.begin(), h.end()), h.end());
        for (int64_t i = s0; i < s1; ++i)
            for (int n = 0; n < 3; ++n) {
                const int32_t code = nbr[n * K + i];
                if (code < 0) continue;
                const int64_t k2 = code >> 2;
                if (k2 >= s0 && k2 < s1) {
                    o.slot[n * K + i] = (int32_t)(k2 - s0);
                } else {
                    const int64_t pos = std::lower_bound(h.begin(), h.end(), (int32_t)k2) - h.begin();
                    o.slot[n * K + i] = (int32_t)(TE + pos);
                }
            }
        // neighbours of the halo triangles: their slot if they are resident (tile or
        // halo), -1 on the boundary, -2 if they lie outside the tile's slots
        for (int32_t e : h)
            for (int n = 0; n < 3; ++n) {
                const int32_t code = nbr[n * K + e];
                int32_t sl = -1;
                if (code >= 0) {
                    const int64_t k2 = code >> 2;
                    if (k2 >= s0 && k2 < s1) {
                        sl = (int32_t)(k2 - s0);
                    } else {
                        auto it = std::lower_bound(h.begin(), h.end(), (int32_t)k2);
                        sl = (it != h.end() && *it == k2) ? (int32_t)(TE + (it - h.begin())) : -2;
                    }
                }
                o.halo_slot.push_back(sl);
            }
        o.halo.insert(o.halo.end(), h.begin(), h.end());
        o.halo_ptr[t + 1] = (int32_t)o.halo.size();
        o.max_halo = std::max<int>(o.max_halo, (int)h.size());
    }
}

void order_and_tile(const double *coordV, const int32_t *V0T, int64_t K, const std::vector<double> &B_usr,
                    const std::vector<int32_t> &nbr_usr, int TE, MeshOrder &o) {
    order_mesh(coordV, V0T, K, B_usr, nbr_usr, o);
    tile_mesh(o.nbr, K, TE, o);
}

int tile_size(int64_t K, int resident, int sms) {
    // tiles of at most 256 triangles; while tiles of 256 leave SMs idle, keep them (one
    // block per SM), else as many as fill a whole number of waves of `resident` blocks,
    // rounded up to whole warps
    if ((K + 255) / 256 <= std::max(1, sms)) return 256;
    const int64_t R = std::max(1, resident);
    const int64_t waves = (K + 256 * R - 1) / (256 * R);
    int64_t te = (K + waves * R - 1) / (waves * R);
    te = ((te + 31) / 32) * 32;
    return (int)std::min<int64_t>(256, std::max<int64_t>(32, te));
}

}  // namespace festung
