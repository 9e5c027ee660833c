// Build step: writes the FP32 reference tables of every supported (p, quadrature) pair
// as initialised device constants (festung_tables_gen.h), from the same build_tables()
// that the library uses at run time.  With the values known to the compiler, every
// table entry in the fused apply becomes an immediate operand of its multiply-add (a
// table read from the constant bank costs an extra load instruction per use on
// sm_103a).  Two sets: the FP32-rounded tables (kind 0) and the BF16-rounded ones
// (kind 1, FESTUNG_BF16TAB).
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "internal.h"

using namespace festung;

namespace {

void emit(FILE *f, const std::vector<double> &v, bool bf16) {
    std::fputs("{", f);
    for (size_t i = 0; i < v.size(); ++i) {
        const float x = bf16 ? round_to_bf16(v[i]) : (float)v[i];
        std::fprintf(f, "%s%.9ef", i ? ", " : "", (double)x);
    }
    std::fputs("}", f);
}

}  // namespace

int main(int argc, char **argv) {
    if (argc != 2) {
        std::fprintf(stderr, "usage: gen_tables OUT.h\n");
        return 2;
    }
    // (p, triangle degree) of every (N, R2, R1) instantiation of the kernels (dispatch.h)
    const struct {
        int p, q, N, R2, R1;
    } cfg[] = {{0, 1, 1, 1, 1},  {1, 2, 3, 3, 2},   {1, 3, 3, 6, 2},   {2, 4, 6, 6, 3},
               {2, 5, 6, 7, 3}, {3, 6, 10, 12, 4}, {3, 7, 10, 16, 4}, {4, 8, 15, 25, 5}};
    FILE *f = std::fopen(argv[1], "w");
    if (!f) return 1;
    std::fputs("// Generated by gen_tables at build time; do not edit.\n#pragma once\n\nnamespace festung {\n", f);
    for (const auto &c : cfg) {
        HostTables T;
        build_tables(c.p, c.q, T);
        if (T.N != c.N || T.R2 != c.R2 || T.R1 != c.R1) {
            std::fprintf(stderr, "gen_tables: p = %d, q = %d gives (%d, %d, %d)\n", c.p, c.q, T.N, T.R2, T.R1);
            return 1;
        }
        for (int kind = 0; kind < 2; ++kind) {
            const char *pre = kind ? "b" : "f";
            std::fprintf(f, "static __device__ const CTab<float, %d, %d, %d> g_%stab_%d_%d_%d = {\n", c.N, c.R2,
                         c.R1, pre, c.N, c.R2, c.R1);
            const std::vector<double> *parts[] = {&T.phiQ, &T.gw1, &T.gw2, &T.H1, &T.H2, &T.phiE, &T.wphiE};
            for (int k = 0; k < 7; ++k) {
                emit(f, *parts[k], kind == 1);
                std::fputs(k < 6 ? ",\n" : "\n", f);
            }
            std::fputs("};\n", f);
            std::fprintf(f,
                         "template <> struct GenTab<%d, %d, %d, %d> {\n"
                         "    static __device__ __forceinline__ const CTab<float, %d, %d, %d> &get() { return "
                         "g_%stab_%d_%d_%d; }\n};\n",
                         c.N, c.R2, c.R1, kind, c.N, c.R2, c.R1, pre, c.N, c.R2, c.R1);
        }
    }
    std::fputs("}  // namespace festung\n", f);
    return std::fclose(f) == 0 ? 0 : 1;
}
