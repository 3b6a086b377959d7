"""Speed-of-light memory model of Sec. 4 (Tables 1-4) and the algorithmic bytes of this library's kernels.

Sec. 4 estimates an operator's best time as (bytes that must cross the memory bus) / (bandwidth) and
its throughput as DoF / time.  ``paper_*`` reproduce the paper's tables for a mesh of E elements and
N nodes (the paper uses E = 1e6, N = 1,030,301); ``kernel_*`` give the algorithmic bytes of one launch
of this library's kernels, which ``bench.py`` divides by the measured kernel time for the roofline.
All sizes are in bytes; MB = 1e6 bytes as in the paper.
"""
from __future__ import annotations

F64 = 8
I32 = 4


# ------------------------------------------------------------------------------ the paper's model ----

def paper_spmv(n_nodes: int, ndpn: int, nnz_per_row: int | None = None, vectors: int = 2) -> dict:
    """Table 1: CSR SpMV.  12 bytes per non-zero (8-byte value + 4-byte column index); ``vectors``
    passes over a DoF vector (the paper's Laplace column counts 2, its mechanics total 3)."""
    rows = n_nodes * ndpn
    nnzr = 27 * ndpn if nnz_per_row is None else nnz_per_row
    matrix = rows * nnzr * (F64 + I32)
    vec = vectors * rows * F64
    return dict(rows=rows, nnz_per_row=nnzr, matrix=matrix, vectors=vec, total=matrix + vec)


def paper_matrix_free(n_elem: int, n_nodes: int, ndpn: int, cell_constants: int) -> dict:
    """Table 2: matrix-free operator.  (perfect caching, no caching) ranges: every nodal value read
    once, or once per element that touches it (8 per element).  The in/out vectors are counted as 3
    passes (read x, read y, write y)."""
    node_map = n_elem * 8 * I32
    cells = n_elem * cell_constants * F64
    pos = (n_nodes * 3 * F64, n_elem * 8 * 3 * F64)
    io = (3 * n_nodes * ndpn * F64, 3 * n_elem * 8 * ndpn * F64)
    tot = tuple(node_map + cells + p + v for p, v in zip(pos, io))
    return dict(node_map=node_map, cell_constants=cells, positions=pos, vectors=io, total=tot)


def paper_partial_assembly(n_elem: int, n_nodes: int, ndpn: int, values_per_qp: int, n_qp: int = 8) -> dict:
    """Table 3: partial assembly (CEED): ``values_per_qp`` stored doubles per quadrature point (6 for
    Laplace, 21 for elasticity).  The printed totals leave out the cell constants."""
    node_map = n_elem * 8 * I32
    qstore = n_elem * n_qp * values_per_qp * F64
    io = (3 * n_nodes * ndpn * F64, 3 * n_elem * 8 * ndpn * F64)
    tot = tuple(node_map + qstore + v for v in io)
    return dict(node_map=node_map, quadrature=qstore, vectors=io, total=tot)


def paper_cg_op(n_nodes: int, ndpn: int) -> int:
    """Table 4: each CG vector operation counted as two vector passes."""
    return 2 * n_nodes * ndpn * F64


def sol_throughput(n_dof: int, bytes_: float, bandwidth_Bps: float) -> float:
    """DoF per second at the speed of light."""
    return n_dof / (bytes_ / bandwidth_Bps)


# ------------------------------------------------------------------- this library's kernels ----

def kernel_apply_bytes(physics: str, n_elem: int, n_nodes: int, structured: bool, real_bytes: int = F64,
                       nrhs: int = 1, tensor_product: bool = False) -> int:
    """Algorithmic (read-once) bytes of one operator apply y = A x.

    Reads: connectivity (unless implicit on a structured box), node coordinates (FP64; on a
    tensor-product grid only the per-axis spacings, which are negligible), one cell constant
    (Laplace kappa) or two (elasticity) stored as 8-byte values, x, the Dirichlet mask (1 byte per
    node); writes y.  ``real_bytes`` is the width of x and y (8 for FP64, 4 for FP32)."""
    ndpn = 1 if physics == "laplace" else 3
    conn = 0 if structured else n_elem * 8 * I32
    coords = 0 if tensor_product else n_nodes * 3 * F64
    cells = n_elem * (1 if physics == "laplace" else 2) * F64
    mask = n_nodes
    vec = 2 * nrhs * n_nodes * ndpn * real_bytes
    return conn + coords + cells + mask + vec


def kernel_spmv_bytes(n_rows: int, nnz: int) -> int:
    """Algorithmic bytes of one CSR SpMV: values + column indices + row pointers + x (read once) + y."""
    return nnz * (F64 + I32) + (n_rows + 1) * I32 + 2 * n_rows * F64


# ------------------------------------------------------ arithmetic of the double-word kernels ----

# FP32-pipe lane operations of the double-word (DW) building blocks (add, sub, mul, fma or integer op
# = one operation each): lazy DW add/sub = TwoSum (6) + 2 adds of the low parts; DW mul = product,
# its FMA error term and two cross FMAs; split of a double into a pair (integer path) and the
# conversion back (exact float-to-double by bits for both parts, one FP64 add).
DW_ADD, DW_MUL, DW_SPLIT, DW_OUT = 8, 4, 12, 13


def kernel_apply_ops(physics: str) -> dict:
    """Algorithmic FP32-pipe operations per element of the face-marching DW apply (one right-hand
    side, tensor-product mesh), counted from the algorithm, not from the compiled code.

    Laplace (one component): 2D transform of the new top face (8 DW adds), z butterfly of the 7
    non-constant modes (7 adds), element coefficients from kappa and the spacings (9 DW muls + 4 DW
    adds + 6 FP32 scalings), diagonal scaling (7 muls), transposed z butterfly with the carried face
    (10 adds), transposed face transform (8 adds), in-plane sums (3 adds), one split in and one
    conversion out per node.
    Elasticity (three components): 3 x (8 + 7) transform adds, coefficients (24 DW muls + 1 DW add +
    26 FP32 scalings), diagonal blocks (12 adds + 33 muls), 24 cross-component multiply-adds,
    3 x (10 + 8 + 3) transposed-transform adds, three splits and three conversions per node."""
    if physics == "laplace":
        parts = {"face_transform": 8 * DW_ADD, "z_butterfly": 7 * DW_ADD, "coefficients": 9 * DW_MUL + 4 * DW_ADD + 6,
                 "scaling": 7 * DW_MUL, "transposed": (10 + 8 + 3) * DW_ADD, "conversions": DW_SPLIT + DW_OUT}
    else:
        parts = {"face_transform": 3 * 8 * DW_ADD, "z_butterfly": 3 * 7 * DW_ADD,
                 "coefficients": 24 * DW_MUL + DW_ADD + 26, "diagonal": 12 * DW_ADD + 33 * DW_MUL,
                 "cross": 24 * (DW_MUL + DW_ADD), "transposed": 3 * (10 + 8 + 3) * DW_ADD,
                 "conversions": 3 * (DW_SPLIT + DW_OUT)}
    return dict(parts=parts, total=sum(parts.values()))


def fp32_lane_peak(sms: int = 152, lanes: int = 128, clock_hz: float = 2.07e9) -> float:
    """FP32-pipe lane operations per second: SMs x FP32 lanes per SM x maximum SM clock."""
    return sms * lanes * clock_hz


# ------------------------------------------------ FP64 arithmetic of the P1 and Q2 kernels ----

def tet_apply_flops(physics: str) -> dict:
    """FP64 operations per P1 tetrahedron of the reference apply (csrc/mf_tet.cuh), a multiply-add
    counted as 2.  Geometry: 9 edge differences, 3 cross products (6 mul + 3 add), n_0 (6 adds),
    D (3 mul + 2 add).  Laplace: 3 differences u_k - u_0, t (3 x (3 mul + 2 add)), c = kappa / (6 D)
    (2), v (4 x (3 mul + 2 add + 1 mul)), 4 scatter adds.  Elasticity: 9 differences, H (9 x (3 mul
    + 2 add)), tr (2), S (9 x 2 + 4), c (2), v (12 x 6), 12 scatter adds."""
    geometry = 9 + 3 * 9 + 6 + 5
    if physics == "elasticity":
        parts = {"geometry": geometry, "gradient": 9 + 9 * 5, "stress": 2 + 9 * 2 + 4 + 2, "scatter": 12 * 6 + 12}
    else:
        parts = {"geometry": geometry, "gradient": 3 + 3 * 5, "flux": 2, "scatter": 4 * 6 + 4}
    return dict(parts=parts, total=sum(parts.values()))


def q2_apply_flops(physics: str, partial_assembly: bool = False) -> dict:
    """FP64 operations per Q2 hexahedron (27 nodes, 27 Gauss points; csrc/mf_q2.cuh), a
    multiply-add counted as 2.

    Reference kernel, per Gauss point: reference gradients of the 27 nodes from the 1D tables (6
    mul each) and J (27 x 9 multiply-adds) = 648; adj J and det J 32; the gradient of u (27 x 3
    multiply-adds per component, 324 or 648 with the gradients reused); the flux (Laplace, 40) or
    the stress (elasticity, 150); the scatter (27 x 3 multiply-adds per component, 324 or 648).
    Partial assembly with sum factorisation: 16 one-dimensional contractions of 27 x 3 multiply-adds
    per component; per Gauss point the flux D_q g_q (Laplace, 9 multiply-adds), or for elasticity
    grad u = H K and P = S K^T (27 multiply-adds each) and the stress S (9 multiply-adds for the
    symmetric part, 2 adds and a multiply for the trace, 3 adds on the diagonal)."""
    if partial_assembly:
        if physics == "elasticity":
            parts = {"contractions": 3 * 2 * 16 * 81, "gradient": 27 * 2 * 27, "stress": 27 * (2 * 9 + 3 + 3),
                     "back": 27 * 2 * 27}
        else:
            parts = {"contractions": 2 * 16 * 81, "flux": 2 * 27 * 9}
    elif physics == "elasticity":
        parts = {"jacobian": 27 * 648, "adjugate": 27 * 32, "gradient": 27 * 648, "stress": 27 * 150,
                 "scatter": 27 * 648}
    else:
        parts = {"jacobian": 27 * 648, "adjugate": 27 * 32, "gradient": 27 * 324, "flux": 27 * 40,
                 "scatter": 27 * 324}
    return dict(parts=parts, total=sum(parts.values()))
