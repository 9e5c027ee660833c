// Compile-time instantiation set of the operator kernels.
#pragma once

#include <type_traits>

namespace festung {

template <int V>
using Int = std::integral_constant<int, V>;

// The supported (N, R2, R1) triples: triangle rule of degree 2p or 2p + 1 and Gauss
// rule exact to degree max(qT, 2p + 1), for p = 0..4.  f is called with three
// integral constants; returns false for an unsupported triple.
template <typename F>
bool dispatch(int N, int R2, int R1, F &&f) {
    if (N == 1 && R2 == 1 && R1 == 1) { f(Int<1>{}, Int<1>{}, Int<1>{}); return true; }
    if (N == 3 && R2 == 3 && R1 == 2) { f(Int<3>{}, Int<3>{}, Int<2>{}); return true; }
    if (N == 3 && R2 == 6 && R1 == 2) { f(Int<3>{}, Int<6>{}, Int<2>{}); return true; }
    if (N == 6 && R2 == 6 && R1 == 3) { f(Int<6>{}, Int<6>{}, Int<3>{}); return true; }
    if (N == 6 && R2 == 7 && R1 == 3) { f(Int<6>{}, Int<7>{}, Int<3>{}); return true; }
    if (N == 10 && R2 == 12 && R1 == 4) { f(Int<10>{}, Int<12>{}, Int<4>{}); return true; }
    if (N == 10 && R2 == 16 && R1 == 4) { f(Int<10>{}, Int<16>{}, Int<4>{}); return true; }
    if (N == 15 && R2 == 25 && R1 == 5) { f(Int<15>{}, Int<25>{}, Int<5>{}); return true; }
    return false;
}

}  // namespace festung
