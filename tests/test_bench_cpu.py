"""The per-unit figures behind bench.py's roofline (no GPU): algorithmic bytes and FLOPs
of one apply per triangle for the two apply workloads, and the counts of quadrature
points they use."""
import bench
import workloads as W


def test_per_triangle_figures_of_the_apply_workloads():
    # 256 x 256, p = 4: N = 15, degree-8 rule with 25 points, 5 Gauss points per edge
    assert bench.bytes_per_element(15, 4, 4) == 208        # FP32 x, D, y + FP32 geometry + neighbour words
    assert bench.bytes_per_element(15, 8, 8) == 404        # FP64
    # contravariant form, multiply-adds counted twice: x traces 225, nonzero H^ entries 2 x 85,
    # edge tests 225, P, Q, zeta 60, d_h and nu.zeta traces 450, volume 25 (45 + 28), edge
    # terms 225, y 30 -> 3210 multiply-adds; 185 single operations
    assert bench.flops_per_element(15, 25, 5) == 2 * 3210 + 185
    # 1024 x 1024, p = 2: N = 6, degree-4 rule with 6 points, 3 Gauss points per edge
    assert bench.bytes_per_element(6, 4, 4) == 100
    # 54 + 2 x 11 + 54 + 24 + 108 + 6 (18 + 10) + 54 + 12 = 496 multiply-adds, 81 single
    assert bench.flops_per_element(6, 6, 3) == 2 * 496 + 81


def test_apply_workloads_are_the_named_configurations():
    c = W.CONFIGS["jitter256_p4"]
    assert (c["n"], c["p"], c["dt"]) == (256, 4, 1e-3)
    c = W.CONFIGS["grf1024_p2"]
    assert (c["n"], c["p"], c["dt"]) == (1024, 2, 1e-4)
    assert bench.CFG_NAME == "jitter256_p4" and bench.APPLY_CFG == "grf1024_p2"


def test_quadrature_counts_of_the_figures():
    from oracle import quadrature
    assert len(quadrature.triangle_rule(8)[0]) == 25 and quadrature.edge_points_for_degree(9) == 5   # p = 4
    assert len(quadrature.triangle_rule(4)[0]) == 6 and quadrature.edge_points_for_degree(5) == 3    # p = 2
