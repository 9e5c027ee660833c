// Internal declarations of the festung library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/festung.h"

namespace festung {

constexpr int PMAX = 4;
constexpr int NMAX = 15;
constexpr int R2MAX = 25;
constexpr int R1MAX = 5;

struct Rule2D {
    std::vector<double> x1, x2, w;
};
struct Rule1D {
    std::vector<double> s, w;
};

int num_dofs(int p);
int edge_points_for_degree(int q);
Rule2D triangle_rule(int q);
Rule1D gauss_legendre01(int n);
void basis_eval(int N, double x1, double x2, double *phi, double *d1, double *d2);

// Reference tables for one (p, quadrature) choice; row-major as indexed.
struct HostTables {
    int p = -1, N = 0, R2 = 0, R1 = 0, qT = 0;
    Rule2D tri;
    Rule1D edge;
    std::vector<double> phiQ;   // [R2][N]  phi_j(q_r)
    std::vector<double> wphiQ;  // [R2][N]  w_r phi_j(q_r)
    std::vector<double> gw1;    // [R2][N]  w_r d_1 phi_i(q_r)
    std::vector<double> gw2;    // [R2][N]  w_r d_2 phi_i(q_r)
    std::vector<double> H1;     // [N][N]   int d_1 phi_i phi_j
    std::vector<double> H2;     // [N][N]   int d_2 phi_i phi_j
    std::vector<double> phiE;   // [3][R1][N] phi_j(gamma_n(s_r))
    std::vector<double> wphiE;  // [3][R1][N] w_r phi_i(gamma_n(s_r))
};
void build_tables(int p, int qT, HostTables &T);
// v rounded to the nearest BF16 value (8-bit significand, ties to even), as a float.
float round_to_bf16(double v);

// Mesh build (host): validates and produces SoA geometry and neighbour codes.
// nbr code of local edge (k, n): interior (k+ << 2) | n+, Dirichlet -1, Neumann -2.
int build_mesh(const double *coordV, int64_t numV, const int32_t *V0T, int64_t numT,
               const int8_t *bdr, std::vector<double> &B /*4 x K*/, std::vector<int32_t> &nbr /*3 x K*/,
               std::string &err);

// Internal element order and tiling (see order_and_tile in mesh.cpp).
struct MeshOrder {
    std::vector<int32_t> perm;      // internal index -> caller's triangle index
    std::vector<int32_t> inv;       // caller's index -> internal index
    std::vector<double> B;          // 4 x K geometry, internal order
    std::vector<int32_t> nbr;       // 3 x K neighbour codes with internal indices
    int TE = 0;                     // triangles per tile
    int max_halo = 0;               // largest halo of any tile
    std::vector<int32_t> halo_ptr;  // tile t's halo is halo[halo_ptr[t] .. halo_ptr[t+1])
    std::vector<int32_t> halo;      // internal indices
    std::vector<int32_t> slot;      // 3 x K: shared-memory slot of the neighbour across edge n (-1: boundary)
    std::vector<int32_t> halo_slot; // 3 per halo entry: slot of its neighbour, -1 boundary, -2 not resident
    std::vector<uint8_t> lift;      // K: bit 1 set if the Dirichlet lift reaches the triangle's right-hand side
};
// order_mesh: perm, inv, B, nbr and lift; tile_mesh: tiles of TE triangles (internal
// neighbour codes nbr) into o's tile fields.
void order_mesh(const double *coordV, const int32_t *V0T, int64_t K, const std::vector<double> &B_usr,
                const std::vector<int32_t> &nbr_usr, MeshOrder &o);
void tile_mesh(const std::vector<int32_t> &nbr, int64_t K, int TE, MeshOrder &o);
// Dirichlet-lift flags (MeshOrder::lift) from internal neighbour codes.
void lift_flags(const std::vector<int32_t> &nbr, int64_t K, std::vector<uint8_t> &lift);
void order_and_tile(const double *coordV, const int32_t *V0T, int64_t K, const std::vector<double> &B_usr,
                    const std::vector<int32_t> &nbr_usr, int TE, MeshOrder &o);
// Tile size (32..256, a multiple of 32) for K triangles when `resident` blocks run at
// once on `sms` multiprocessors.
int tile_size(int64_t K, int resident, int sms);

// Device-side view passed to kernels.
template <typename T>
struct DevMesh {
    const T *B;          // 4 x K: B11, B12, B21, B22
    const int32_t *nbr;  // 3 x K
    int64_t K;
};

// Device table buffer in the layout of kernels (one contiguous block per precision).
struct TableOffsets {
    int phiQ, wphiQ, gw1, gw2, H1, H2, phiE, wphiE, total;
};
TableOffsets table_offsets(int N, int R2, int R1);

struct Workspace;  // Krylov vectors
struct dfloat;     // double-float value (dfloat.cuh)

}  // namespace festung

struct festung_ctx {
    int64_t K = 0, numV = 0;
    std::vector<double> coordV;
    std::vector<int32_t> V0T;
    std::vector<int8_t> bdr;
    std::vector<double> hB;  // 4 x K geometry in the caller's triangle order
    std::vector<int32_t> perm;  // internal index -> caller's triangle index
    int32_t *dPerm = nullptr;   // device copy of perm
    int TE = 0, max_halo = 0, nslot = 0;
    int fthreads = 320;  // threads of a fused-apply block: TE plus whole warps for the halo
    std::vector<int32_t> hNbrInt;  // 3 x K neighbour codes in internal order (for re-tiling)
    int32_t *dHaloPtr = nullptr, *dHalo = nullptr;
    int16_t *dSlot = nullptr;   // 3 x K
    int16_t *dHaloSlot = nullptr;  // 3 per halo entry
    uint8_t *dLift = nullptr;      // K, see MeshOrder::lift
    int32_t *dLiftList = nullptr;  // the triangles whose right-hand side the Dirichlet lift reaches
    int64_t nLift = 0;
    bool has_dirichlet = false, has_neumann = false;
    // device mesh
    double *dB = nullptr;
    float *fB = nullptr;
    int32_t *dNbr = nullptr;
    // order / tables
    int p = -1, N = 0, R2 = 0, R1 = 0, qT = 0;
    double eta = 1.0;
    double mass = 1.0;  // coefficient of M in the operator: 1 for a step, 0 for the stationary problem
    festung::HostTables tab;
    double *dTab = nullptr;  // FP64 tables, layout table_offsets
    float *fTab = nullptr;   // FP32 copy
    float *bTab = nullptr;   // BF16-rounded values (FESTUNG_BF16TAB), FP32 storage
    bool tab_bf16 = false;   // FP32 applies use the BF16-rounded tables (set during such solves)
    // state and data (N x K unless noted)
    double *dC = nullptr, *dD = nullptr, *dF = nullptr;
    double *dCprev = nullptr, *dCprev2 = nullptr;  // C^{n-1}, C^{n-2} for the extrapolated initial guess
    int hist = 0;                                  // number of valid previous states (0..2)
    uint64_t state_gen = 0;                        // bumped whenever C changes (batches detect outside changes)
    double *dGuess = nullptr;                      // N x K correction of the next step's initial guess
    bool has_guess = false;                        // dGuess holds a guess for the next step
    festung_ctx *coarse = nullptr;                 // the p = 1 problem on the same mesh (coarse correction)
    int coarse_mode = 0;                           // 1: each FP32 sweep starts from a coarse correction
    bool coarse_warm = false;                      // the coarse context's x holds the last coarse solution
    double dt_prev = 0.0, dt_prev2 = 0.0;
    float *fD = nullptr;
    // double-float copies for the residual of the mixed-precision refinement
    festung::dfloat *xD = nullptr;    // N x K, refreshed from dD when xD_valid is false
    festung::dfloat *xB = nullptr;    // 4 x K geometry
    festung::dfloat *xTab = nullptr;  // tables, layout table_offsets
    bool xD_valid = false;
    double *dCD = nullptr, *dGN = nullptr;  // K x 3 x R1 boundary samples
    double *dSamp = nullptr;                // K x R2 staging for projections
    bool symmetric = true;
    bool source_zero = true;
    bool bc_zero = true;
    // workspace
    festung::Workspace *ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;         // the preconditioner build overlaps the right-hand side and residual
    cudaEvent_t ev_in = nullptr, ev_P = nullptr;
    bool P_pending = false;              // the block-Jacobi build runs on `side` until ev_P
    // reuse of the block-Jacobi blocks over steps (festung_set_precond_reuse)
    int precond_reuse = 1;     // steps one build serves at most (1: every step builds its own)
    bool P_valid = false;      // w.P / w.Pb hold blocks of S for P_dt and P_mass
    double P_dt = 0.0, P_mass = -1.0;
    int P_age = 0;             // steps served by the current blocks
    int P_iters0 = -1;         // Krylov iterations of the step that built them
    bool P_built = false;      // the current step built its blocks
    bool persistent = true;    // FP32 BiCGStab at p <= 1 as one persistent kernel (festung_set_persistent)
    bool persist_refused = false;  // the device refused the persistent grid once: the graph form
    int test_barrier_extra = 0;    // festung_test_barrier_timeout: barriers wait for this many more blocks
    int num_sms = 0;
    mutable int64_t launches = 0;  // kernels launched on behalf of this context (graph nodes counted)
    std::string err;
};
