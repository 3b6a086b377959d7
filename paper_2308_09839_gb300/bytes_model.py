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
