"""The speed-of-light byte model reproduces the paper's Tables 1-4 (tests/golden/paper_tables.json)."""
import json
import os

import pytest

from paper_2308_09839_gb300 import bytes_model as bm

T = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
E, N = T["n_elem"], T["n_nodes"]
MB = 1e6


def close(a, b, rel=0.03, abs_=0.6):
    return abs(a - b) <= max(rel * abs(b), abs_)


def test_table1_spmv():
    lap = bm.paper_spmv(N, 1)
    mech = bm.paper_spmv(N, 3, vectors=3)
    t = T["table1_spmv"]
    assert lap["rows"] == t["laplace"]["rows"] and mech["rows"] == t["mechanics"]["rows"]
    assert close(lap["matrix"] / MB, 333.8, abs_=0.1)  # printed 343 (see _readings)
    assert close(mech["matrix"] / MB, t["mechanics"]["matrix_MB"])
    assert close(bm.paper_spmv(N, 1)["vectors"] / MB, t["laplace"]["vector_MB"])
    assert close(mech["total"] / MB, t["mechanics"]["total_MB"])
    # implied bandwidths: printed throughput = rows / printed time
    for gpu, (tl, tm) in t["time_ms"].items():
        gl, gm = t["gdofs"][gpu]
        assert close(lap["rows"] / (tl * 1e-3) / 1e9, gl, rel=0.05)
        assert close(mech["rows"] / (tm * 1e-3) / 1e9, gm, rel=0.08)


@pytest.mark.parametrize("phys,ndpn,cc", [("laplace", 1, 0), ("elasticity", 3, 2)])
def test_table2_matrix_free(phys, ndpn, cc):
    m = bm.paper_matrix_free(E, N, ndpn, cc)
    t = T["table2_matrix_free"][phys]
    assert close(m["node_map"] / MB, t["node_map_MB"])
    assert close(m["cell_constants"] / MB, t["cell_constant_MB"])
    for k in range(2):
        assert close(m["positions"][k] / MB, t["positions_MB"][k])
        assert close(m["vectors"][k] / MB, t["vectors_MB"][k])
        assert close(m["total"][k] / MB, t["total_MB"][k], abs_=1.0)


def test_table2_throughput_ranges():
    """Throughput = DoF / (total / bandwidth) with the bandwidth implied by Table 1."""
    t = T["table2_matrix_free"]["gdofs"]
    for gpu, (tl, _) in T["table1_spmv"]["time_ms"].items():
        bw = 359e6 / (tl * 1e-3)
        for (phys, ndpn, cc), (hi, lo) in zip([("laplace", 1, 0), ("elasticity", 3, 2)], t[gpu]):
            m = bm.paper_matrix_free(E, N, ndpn, cc)
            assert close(bm.sol_throughput(N * ndpn, m["total"][0], bw) / 1e9, hi, rel=0.12)
            assert close(bm.sol_throughput(N * ndpn, m["total"][1], bw) / 1e9, lo, rel=0.12)


@pytest.mark.parametrize("phys,ndpn,v", [("laplace", 1, 6), ("elasticity", 3, 21)])
def test_table3_partial_assembly(phys, ndpn, v):
    m = bm.paper_partial_assembly(E, N, ndpn, v)
    t = T["table3_partial_assembly"][phys]
    assert close(m["quadrature"] / MB, t["quadrature_MB"])
    for k in range(2):
        assert close(m["total"][k] / MB, t["total_MB"][k], abs_=1.5)


def test_table4_cg_ops():
    assert close(bm.paper_cg_op(N, 1) / MB, T["table4_cg_op_MB"]["laplace"], abs_=0.05)
    assert close(bm.paper_cg_op(N, 3) / MB, T["table4_cg_op_MB"]["mechanics"], abs_=0.1)


def test_kernel_bytes_config_sizes():
    """Algorithmic bytes of the 256^3 Cartesian Laplace apply (implicit connectivity)."""
    n = 256
    b = bm.kernel_apply_bytes("laplace", n ** 3, (n + 1) ** 3, structured=True)
    assert b == (n + 1) ** 3 * (24 + 1 + 16) + n ** 3 * 8


def test_kernel_bytes_tensor_product():
    n = 256
    b = bm.kernel_apply_bytes("laplace", n ** 3, (n + 1) ** 3, structured=True, tensor_product=True)
    assert b == (n + 1) ** 3 * (1 + 16) + n ** 3 * 8


def test_p1_q2_operation_counts():
    """The FP64 operation counts the bench divides by for the P1 and Q2 kernels: totals of their
    parts, and the partial assembly's count below the reference kernel's by the expected factor."""
    from paper_2308_09839_gb300 import bytes_model as bm
    assert bm.tet_apply_flops("laplace")["total"] == 95
    assert bm.tet_apply_flops("elasticity")["total"] == 211
    ref = bm.q2_apply_flops("laplace")["total"]
    pa = bm.q2_apply_flops("laplace", partial_assembly=True)["total"]
    assert ref == 36936 and pa == 3078 and 11 < ref / pa < 13
    assert bm.q2_apply_flops("elasticity")["total"] == 57402
    pe = bm.q2_apply_flops("elasticity", partial_assembly=True)["total"]
    assert pe == 3 * 2592 + 2 * 1458 + 648 and 4 < 57402 / pe < 6
