"""The work models behind the bench line's roofline (bench.kernel_work), checked against
their definitions: the flops of each contraction of the right-hand side, the BF16 slice
products the kernels issue for them, and the HBM bytes of the orbit assembly, counted
stage by stage from what each RK4 stage reads and writes per element of G2."""
import pytest

import bench


@pytest.mark.parametrize("nb", [32, 64, 96])
def test_polarisation_work(nb):
    """Pi_(ik),(jl) = sum_(pq) G_ipkq hcorr_qjpl (Eq. gwpi): nb^6 complex multiply-adds, 8 real
    flops each; the kernel runs the realified product (nb^2 rows, 2 nb^2 columns, 2 nb^2 terms)
    with six BF16 slice products per real multiply-add."""
    bound, alg, issued = bench.kernel_work("tc_gemm_pi", nb, "GW", "bf16x4")
    assert bound == "tensor"
    assert alg == 8 * nb ** 6
    assert issued == 2 * 6 * nb ** 2 * (2 * nb ** 2) * (2 * nb ** 2)
    assert issued / alg == pytest.approx(6.0)


@pytest.mark.parametrize("nb", [32, 96])
def test_nb5_pass_work(nb):
    """A complex nb^5 pass (e.g. the commutator Z = G2 x_4 h): nb^5 complex multiply-adds, realified
    as nb^3 rows x 2 nb columns x 2 nb terms with ten BF16 slice products each; a pass with the real
    w as A (source pass 1) has nb terms: nb^5 real-by-complex multiply-adds (4 flops)."""
    _, alg, issued = bench.kernel_work("tc_gemm_commutator", nb, "SOA", "bf16x4")
    assert alg == 8 * nb ** 5
    assert issued == 2 * 10 * nb ** 3 * (2 * nb) * (2 * nb)
    _, alg1, issued1 = bench.kernel_work("tc_gemm_psi1", nb, "SOA", "bf16x4")
    assert alg1 == 4 * nb ** 5
    assert issued1 == 2 * 10 * nb ** 3 * (2 * nb) * nb
    # the collision integral: nb x nb outputs per plane, nb^3 terms, real w
    _, algc, issuedc = bench.kernel_work("tc_gemm_collision", nb, "SOA", "bf16x4")
    assert algc == 4 * nb ** 5
    assert issuedc == 2 * 10 * (2 * nb) * nb * nb ** 3


@pytest.mark.parametrize("se,extra", [("SOA", 0), ("GW", 8)])
def test_assembly_bytes(se, extra):
    """Bytes per element of each stage of the orbit assembly: Z and Q (8 B each, and Pi for GW)
    in every stage; stages 0-2 read the FP32 state copy (8 B) and write the accumulator and the
    next stage input (8 B each), stages 1-2 also read the accumulator (8 B); the last stage reads
    the FP64 state (16 B) and the accumulator, and writes the FP64 state and its FP32 copy."""
    zq = 16 + extra
    stage = [zq + 8 + 8 + 8,            # stage 0: FP32 state; writes accumulator, stage input
             zq + 8 + 8 + 8 + 8,        # stages 1, 2: + accumulator read
             zq + 8 + 8 + 8 + 8,
             zq + 16 + 8 + 16 + 8]      # last stage: FP64 state, accumulator; writes FP64 state, FP32 copy
    per_elem = sum(stage) / 4
    nb = 96
    bound, alg, issued = bench.kernel_work("tc_orbit_assemble_rk4", nb, se, "bf16x4")
    assert bound == "hbm"
    assert alg == pytest.approx(per_elem * nb ** 4)
    assert issued == alg
    assert per_elem == 50 + extra
