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
