"""Thin ctypes binding to ``libmf.so`` (argument marshalling only).

Every function of ``include/mf.h`` is exposed under the same name; tensors are passed as device
pointers (``tensor.data_ptr()``) and the stream defaults to PyTorch's current CUDA stream.  Nothing
here computes: when the library is missing the import fails loudly (no CPU fallback).

``Mesh`` and ``Csr`` are small owners of the opaque handles with the same calls as methods.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

# MF_LIB: path of another build of the library (the bounds-checked libmf_debug.so) to load instead
_LIB_PATH = os.environ.get("MF_LIB") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmf.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is not built; run `python -m paper_2308_09839_gb300.build` "
                      "(or __graft_entry__.build()) first")
lib = C.CDLL(_LIB_PATH)

MF_OK, MF_NOT_CONVERGED = 0, 1
MF_ERR_ARG, MF_ERR_CUDA, MF_ERR_MESH, MF_ERR_OOM, MF_ERR_BREAKDOWN, MF_ERR_TIMEOUT, MF_ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7
MF_LAPLACE, MF_ELASTICITY, MF_VECTOR_LAPLACE = 0, 1, 2
PHYSICS = {"laplace": MF_LAPLACE, "elasticity": MF_ELASTICITY, "vector_laplace": MF_VECTOR_LAPLACE}
MF_VARIANT_AUTO, MF_VARIANT_REFERENCE, MF_VARIANT_GENERAL, MF_VARIANT_PARTIAL = 0, 1, 2, 3
MF_ELEM_HEX8, MF_ELEM_TET4, MF_ELEM_HEX27 = 0, 1, 2
ELEMENTS = {"hex8": MF_ELEM_HEX8, "tet4": MF_ELEM_TET4, "hex27": MF_ELEM_HEX27}
MF_CG_CLASSIC, MF_CG_PIPELINED, MF_CG_CLASSIC_SPLIT = 0, 1, 2
MF_OP_MATFREE, MF_OP_CSR = 0, 1
MF_PREC_FP64, MF_PREC_MIXED_IR = 0, 1
MF_PC_NONE, MF_PC_JACOBI, MF_PC_LEARNED = 0, 1, 2

STATUS_NAMES = {0: "MF_OK", 1: "MF_NOT_CONVERGED", -1: "MF_ERR_ARG", -2: "MF_ERR_CUDA", -3: "MF_ERR_MESH",
                -4: "MF_ERR_OOM", -5: "MF_ERR_BREAKDOWN", -6: "MF_ERR_TIMEOUT", -7: "MF_ERR_UNSUPPORTED"}

vp = C.c_void_p
i32, i64, f64 = C.c_int32, C.c_int64, C.c_double


class mf_solve_opts(C.Structure):
    _fields_ = [("op", i32), ("precision", i32), ("precond", i32), ("max_iter", i32), ("rtol", f64),
                ("check_every", i32), ("use_graph", i32), ("timeout_s", f64), ("inner_rtol", f64),
                ("max_outer", i32), ("csr", vp), ("net", vp), ("recurrence", i32)]


class mf_solve_info(C.Structure):
    _fields_ = [("iters", i32), ("outer_iters", i32), ("status", i32), ("reserved", i32), ("rel_res", f64),
                ("rel_res_true", f64), ("seconds", f64)]


_SIGS = {
    "mf_setup_mesh": (C.c_int, [C.c_int, i64, i64, vp, vp, i32, i32, i32, vp, vp, vp, C.POINTER(vp)]),
    "mf_setup_mesh_elem": (C.c_int, [C.c_int, C.c_int, i64, i64, vp, vp, vp, vp, vp, C.POINTER(vp)]),
    "mf_destroy_mesh": (C.c_int, [vp]),
    "mf_mesh_query": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64),
                                C.POINTER(i32), C.POINTER(i32)]),
    "mf_set_apply_variant": (C.c_int, [vp, C.c_int]),
    "mf_apply_laplace": (C.c_int, [vp, vp, vp, vp]),
    "mf_apply_elasticity": (C.c_int, [vp, vp, vp, vp]),
    "mf_apply_vector_laplace": (C.c_int, [vp, vp, vp, vp]),
    "mf_apply_f32": (C.c_int, [vp, vp, vp, vp]),
    "mf_apply_multi": (C.c_int, [vp, i32, vp, vp, vp]),
    "mf_assemble_csr": (C.c_int, [vp, vp, C.POINTER(vp)]),
    "mf_csr_query": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]),
    "mf_csr_export": (C.c_int, [vp, vp, vp, vp, vp]),
    "mf_spmv_csr": (C.c_int, [vp, vp, vp, vp]),
    "mf_destroy_csr": (C.c_int, [vp]),
    "mf_solve_opts_default": (None, [C.POINTER(mf_solve_opts)]),
    "mf_cg_solve": (C.c_int, [vp, C.POINTER(mf_solve_opts), vp, vp, C.POINTER(mf_solve_info), vp]),
    "mf_cg_solve_noalloc": (C.c_int, [vp, C.POINTER(mf_solve_opts), vp, vp, C.POINTER(mf_solve_info), vp]),
    "mf_cg_state_bytes": (C.c_size_t, [vp]),
    "mf_cg_state_save": (C.c_int, [vp, vp, C.c_size_t, vp]),
    "mf_cg_resume": (C.c_int, [vp, C.POINTER(mf_solve_opts), vp, C.c_size_t, vp, vp, C.POINTER(mf_solve_info), vp]),
    "mf_batch_create": (C.c_int, [C.POINTER(vp), i32, C.POINTER(mf_solve_opts), C.POINTER(vp)]),
    "mf_batch_solve": (C.c_int, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(mf_solve_info), vp]),
    "mf_batch_destroy": (C.c_int, [vp]),
    "mf_cg_solve_batched": (C.c_int, [C.POINTER(vp), i32, C.POINTER(mf_solve_opts), C.POINTER(vp), C.POINTER(vp),
                                      C.POINTER(mf_solve_info), vp]),
    "mf_set_tile_segment": (C.c_int, [vp, i32]),
    "mf_debug_status": (C.c_int, [C.POINTER(C.c_uint32), C.POINTER(i32)]),
    "mf_net_create": (C.c_int, [i32, i32, i32, C.c_uint64, C.POINTER(vp)]),
    "mf_net_destroy": (C.c_int, [vp]),
    "mf_net_num_params": (i64, [vp]),
    "mf_net_get_params": (C.c_int, [vp, vp]),
    "mf_net_set_params": (C.c_int, [vp, vp]),
    "mf_net_state_bytes": (i64, [vp]),
    "mf_net_state_save": (C.c_int, [vp, vp, i64]),
    "mf_net_state_load": (C.c_int, [vp, vp, i64]),
    "mf_net_set_output_scale": (C.c_int, [vp, C.c_float]),
    "mf_net_forward": (C.c_int, [vp, vp, vp, vp, vp]),
    "mf_node_logk": (C.c_int, [vp, vp, vp]),
    "mf_net_train_step": (C.c_int, [vp, vp, vp, vp, C.c_float, C.POINTER(C.c_float), vp]),
    "mf_net_gradients": (C.c_int, [vp, vp, vp, vp, vp, C.POINTER(C.c_float), vp]),
    "mf_conv3d_fwd": (C.c_int, [vp, i32, i32, i32, i32, vp, vp, i32, vp, i32, vp, vp, vp]),
    "mf_conv3d_dgrad": (C.c_int, [vp, i32, i32, i32, i32, vp, i32, vp, vp, vp]),
    "mf_conv3d_wgrad_workspace": (i64, [i32, i32, i32, i32, i32]),
    "mf_conv3d_wgrad": (C.c_int, [vp, vp, i32, i32, i32, i32, i32, vp, vp, vp, i64, vp]),
    "mf_grid_restrict": (C.c_int, [vp, i32, i32, i32, i32, vp, C.c_float, vp]),
    "mf_grid_prolong": (C.c_int, [vp, i32, i32, i32, i32, vp, C.c_float, vp]),
    "mf_operator_diagonal": (C.c_int, [vp, vp, vp]),
    "mf_training_pair": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(C.c_double), vp]),
    "mf_kernel_launches": (i64, []),
    "mf_last_error": (C.c_char_p, []),
    "mf_version": (C.c_char_p, []),
}
EXPORTED = tuple(_SIGS)

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class MfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.mf_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def check(status: int, where: str, ok=(MF_OK,)) -> int:
    if status not in ok:
        raise MfError(status, where)
    return status


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


# ----------------------------------------------------------------------- same-name functions ----

def mf_setup_mesh(physics, n_nodes, n_cells, coords, cells, nx, ny, nz, mat, dirichlet, stream=None) -> int:
    h = vp()
    check(lib.mf_setup_mesh(physics, n_nodes, n_cells, _ptr(coords), _ptr(cells), nx, ny, nz, _ptr(mat),
                            _ptr(dirichlet), _stream(stream), C.byref(h)), "mf_setup_mesh")
    return h.value


def mf_setup_mesh_elem(element, physics, n_nodes, n_cells, coords, cells, mat, dirichlet, stream=None) -> int:
    """Mesh of an explicit connectivity of element type MF_ELEM_HEX8 ([E][8]), MF_ELEM_TET4 ([E][4],
    positively oriented) or MF_ELEM_HEX27 ([E][27], node i + 3j + 9k at reference (i-1, j-1, k-1))."""
    h = vp()
    check(lib.mf_setup_mesh_elem(element, physics, n_nodes, n_cells, _ptr(coords), _ptr(cells), _ptr(mat),
                                 _ptr(dirichlet), _stream(stream), C.byref(h)), "mf_setup_mesh_elem")
    return h.value


def mf_destroy_mesh(h) -> None:
    check(lib.mf_destroy_mesh(h), "mf_destroy_mesh")


def mf_mesh_query(h) -> dict:
    a, b, c, d = i64(), i64(), i64(), i64()
    e, f = i32(), i32()
    check(lib.mf_mesh_query(h, C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(e), C.byref(f)), "mf_mesh_query")
    return dict(n_nodes=a.value, n_cells=b.value, n_dof=c.value, n_free=d.value, n_colours=e.value,
                structured=bool(f.value & 1), all_affine=bool(f.value & 2), tensor_product=bool(f.value & 4),
                partial_assembly=bool(f.value & 8), tetrahedral=bool(f.value & 16), q2=bool(f.value & 32),
                dw_range_exceeded=bool(f.value & 64), dw_normalised=bool(f.value & 128), flags=f.value)


def mf_set_apply_variant(h, variant: int) -> None:
    check(lib.mf_set_apply_variant(h, variant), "mf_set_apply_variant")


def mf_apply_laplace(h, x, y, stream=None) -> None:
    check(lib.mf_apply_laplace(h, _ptr(x), _ptr(y), _stream(stream)), "mf_apply_laplace")


def mf_apply_elasticity(h, x, y, stream=None) -> None:
    check(lib.mf_apply_elasticity(h, _ptr(x), _ptr(y), _stream(stream)), "mf_apply_elasticity")


def mf_apply_vector_laplace(h, x, y, stream=None) -> None:
    check(lib.mf_apply_vector_laplace(h, _ptr(x), _ptr(y), _stream(stream)), "mf_apply_vector_laplace")


def mf_apply_f32(h, x, y, stream=None) -> None:
    check(lib.mf_apply_f32(h, _ptr(x), _ptr(y), _stream(stream)), "mf_apply_f32")


def mf_apply_multi(h, nrhs, X, Y, stream=None) -> None:
    check(lib.mf_apply_multi(h, nrhs, _ptr(X), _ptr(Y), _stream(stream)), "mf_apply_multi")


def mf_assemble_csr(h, stream=None) -> int:
    out = vp()
    check(lib.mf_assemble_csr(h, _stream(stream), C.byref(out)), "mf_assemble_csr")
    return out.value


def mf_csr_query(a) -> dict:
    n, z = i64(), i64()
    rp, cl, vl = vp(), vp(), vp()
    check(lib.mf_csr_query(a, C.byref(n), C.byref(z), C.byref(rp), C.byref(cl), C.byref(vl)), "mf_csr_query")
    return dict(n_rows=n.value, nnz=z.value, rowptr=rp.value, col=cl.value, val=vl.value)


def mf_csr_export(a, rowptr, col, val, stream=None) -> None:
    check(lib.mf_csr_export(a, _ptr(rowptr), _ptr(col), _ptr(val), _stream(stream)), "mf_csr_export")


def mf_spmv_csr(a, x, y, stream=None) -> None:
    check(lib.mf_spmv_csr(a, _ptr(x), _ptr(y), _stream(stream)), "mf_spmv_csr")


def mf_destroy_csr(a) -> None:
    check(lib.mf_destroy_csr(a), "mf_destroy_csr")


def mf_solve_opts_default() -> mf_solve_opts:
    o = mf_solve_opts()
    lib.mf_solve_opts_default(C.byref(o))
    return o


def mf_cg_solve(h, opts: mf_solve_opts, b, x, stream=None, ok=(MF_OK, MF_NOT_CONVERGED)) -> mf_solve_info:
    info = mf_solve_info()
    st = lib.mf_cg_solve(h, C.byref(opts), _ptr(b), _ptr(x), C.byref(info), _stream(stream))
    check(st, "mf_cg_solve", ok)
    return info


def mf_cg_solve_noalloc(h, opts: mf_solve_opts, b, x, stream=None, ok=(MF_OK, MF_NOT_CONVERGED)) -> mf_solve_info:
    """CG whose scratch is a fixed array inside the library (no device allocation; n_dof <=
    MF_NOALLOC_MAX_DOF)."""
    info = mf_solve_info()
    st = lib.mf_cg_solve_noalloc(h, C.byref(opts), _ptr(b), _ptr(x), C.byref(info), _stream(stream))
    check(st, "mf_cg_solve_noalloc", ok)
    return info


MF_NOALLOC_MAX_DOF = 262144


def mf_cg_state_bytes(h) -> int:
    return int(lib.mf_cg_state_bytes(h))


def mf_cg_state_save(h, stream=None) -> bytes:
    """The checkpoint of the last stopped classic FP64 CG solve on this mesh, as bytes."""
    n = mf_cg_state_bytes(h)
    buf = C.create_string_buffer(n)
    check(lib.mf_cg_state_save(h, buf, n, _stream(stream)), "mf_cg_state_save")
    return buf.raw


def mf_cg_resume(h, opts: mf_solve_opts, state: bytes, b, x, stream=None, ok=(MF_OK, MF_NOT_CONVERGED)) -> mf_solve_info:
    info = mf_solve_info()
    buf = C.create_string_buffer(state, len(state))
    st = lib.mf_cg_resume(h, C.byref(opts), buf, len(state), _ptr(b), _ptr(x), C.byref(info), _stream(stream))
    check(st, "mf_cg_resume", ok)
    return info


def _vec(t, n: int, dtypes, what: str) -> None:
    """Refuse a vector that the kernels would read or write out of bounds: a dtype other than the
    ones the call takes, or fewer than n elements."""
    if t.dtype not in dtypes:
        raise ValueError(f"{what}: dtype {t.dtype}; expected {' or '.join(str(d) for d in dtypes)}")
    if t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements; {n} needed")


def _ptr_array(ts):
    arr = (vp * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _ptr(t)
    return arr


def mf_batch_create(meshes, opts: mf_solve_opts) -> int:
    hs = (vp * len(meshes))(*[m.h if isinstance(m, Mesh) else m for m in meshes])
    out = vp()
    check(lib.mf_batch_create(hs, len(meshes), C.byref(opts), C.byref(out)), "mf_batch_create")
    return out.value


def mf_batch_solve(batch, bs, xs, stream=None, ok=(MF_OK, MF_NOT_CONVERGED)):
    infos = (mf_solve_info * len(bs))()
    st = lib.mf_batch_solve(batch, _ptr_array(bs), _ptr_array(xs), infos, _stream(stream))
    check(st, "mf_batch_solve", ok)
    return list(infos)


def mf_batch_destroy(batch) -> None:
    check(lib.mf_batch_destroy(batch), "mf_batch_destroy")


def mf_cg_solve_batched(meshes, opts: mf_solve_opts, bs, xs, stream=None, ok=(MF_OK, MF_NOT_CONVERGED)):
    hs = (vp * len(meshes))(*[m.h if isinstance(m, Mesh) else m for m in meshes])
    infos = (mf_solve_info * len(bs))()
    st = lib.mf_cg_solve_batched(hs, len(meshes), C.byref(opts), _ptr_array(bs), _ptr_array(xs), infos,
                                 _stream(stream))
    check(st, "mf_cg_solve_batched", ok)
    return list(infos)


def mf_node_logk(mesh, out=None, stream=None):
    """Node mean of log kappa of a scalar Laplace structured box (device float32[n_nodes])."""
    if out is None:
        out = torch.empty(mesh.info["n_nodes"], dtype=torch.float32, device=mesh.device)
    check(lib.mf_node_logk(mesh.h, _ptr(out), _stream(stream)), "mf_node_logk")
    return out


def mf_debug_status() -> tuple[int, bool]:
    """(bits of failed index checks since the last call, whether the loaded library checks at all)."""
    bits, en = C.c_uint32(), i32()
    check(lib.mf_debug_status(C.byref(bits), C.byref(en)), "mf_debug_status")
    return int(bits.value), bool(en.value)


def mf_set_tile_segment(h, seg: int) -> None:
    check(lib.mf_set_tile_segment(h.h if isinstance(h, Mesh) else h, seg), "mf_set_tile_segment")


# ------------------------------------------------------------------ learned preconditioner ----

def _bf16_ptr(t):
    if t is None:
        return None
    assert t.dtype == torch.bfloat16
    return _ptr(t)


def mf_conv3d_fwd(x, w, bias, cout, skip=None, relu=False, y_bf16=None, y_f32=None, stream=None):
    nz, ny, nx, cin = x.shape
    check(lib.mf_conv3d_fwd(_bf16_ptr(x), nx, ny, nz, cin, _bf16_ptr(w), _ptr(bias), cout, _bf16_ptr(skip),
                            int(relu), _bf16_ptr(y_bf16), _ptr(y_f32), _stream(stream)), "mf_conv3d_fwd")


def mf_conv3d_dgrad(dy, w, cin, dx_bf16=None, dx_f32=None, stream=None):
    nz, ny, nx, cout = dy.shape
    check(lib.mf_conv3d_dgrad(_bf16_ptr(dy), nx, ny, nz, cin, _bf16_ptr(w), cout, _bf16_ptr(dx_bf16), _ptr(dx_f32),
                              _stream(stream)), "mf_conv3d_dgrad")


def mf_conv3d_wgrad(x, dy, stream=None):
    nz, ny, nx, cin = x.shape
    cout = dy.shape[3]
    nbytes = int(lib.mf_conv3d_wgrad_workspace(nx, ny, nz, cin, cout))
    ws = torch.empty(nbytes // 4 + 1, dtype=torch.float32, device=x.device)
    dw = torch.empty(27, cin, cout, dtype=torch.float32, device=x.device)
    db = torch.empty(cout, dtype=torch.float32, device=x.device)
    check(lib.mf_conv3d_wgrad(_bf16_ptr(x), _bf16_ptr(dy), nx, ny, nz, cin, cout, _ptr(dw), _ptr(db), _ptr(ws), nbytes,
                              _stream(stream)), "mf_conv3d_wgrad")
    return dw, db


def mf_grid_restrict(x, scale=1.0, stream=None):
    nz, ny, nx, c = x.shape
    out = torch.empty((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2, c, dtype=x.dtype, device=x.device)
    check(lib.mf_grid_restrict(_bf16_ptr(x), nx, ny, nz, c, _bf16_ptr(out), scale, _stream(stream)), "mf_grid_restrict")
    return out


def mf_grid_prolong(x, scale=1.0, stream=None):
    nz, ny, nx, c = x.shape
    out = torch.empty(2 * nz - 1, 2 * ny - 1, 2 * nx - 1, c, dtype=x.dtype, device=x.device)
    check(lib.mf_grid_prolong(_bf16_ptr(x), nx, ny, nz, c, _bf16_ptr(out), scale, _stream(stream)), "mf_grid_prolong")
    return out


class Net:
    """Owner of an ``mf_net`` (the learned preconditioner) for a node grid (nx, ny, nz)."""

    def __init__(self, nx, ny, nz, seed=0):
        h = vp()
        check(lib.mf_net_create(nx, ny, nz, seed, C.byref(h)), "mf_net_create")
        self.h = h.value
        self.dims = (nx, ny, nz)
        self.n_params = int(lib.mf_net_num_params(self.h))

    def params(self):
        import numpy as np
        out = np.empty(self.n_params, dtype=np.float32)
        check(lib.mf_net_get_params(self.h, out.ctypes.data), "mf_net_get_params")
        return out

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        check(lib.mf_net_set_params(self.h, p.ctypes.data), "mf_net_set_params")

    def set_output_scale(self, s):
        check(lib.mf_net_set_output_scale(self.h, float(s)), "mf_net_set_output_scale")

    def state(self):
        """The whole training state (mf_net_state_save) as a uint8 array."""
        import numpy as np
        out = np.empty(int(lib.mf_net_state_bytes(self.h)), dtype=np.uint8)
        check(lib.mf_net_state_save(self.h, out.ctypes.data, out.size), "mf_net_state_save")
        return out

    def load_state(self, blob):
        """Restore a training state taken by state() (mf_net_state_load)."""
        import numpy as np
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        check(lib.mf_net_state_load(self.h, blob.ctypes.data, blob.size), "mf_net_state_load")

    def _fields(self, what, *ts):
        """Node fields of the network's grid: float32, nx ny nz elements each."""
        n = self.dims[0] * self.dims[1] * self.dims[2]
        for name, t in ts:
            _vec(t, n, (torch.float32,), f"Net.{what} {name}")

    def forward(self, r, logk, out=None, stream=None):
        self._fields("forward", ("r", r), ("logk", logk))
        if out is None:
            out = torch.empty_like(r)
        self._fields("forward", ("out", out))
        check(lib.mf_net_forward(self.h, _ptr(r), _ptr(logk), _ptr(out), _stream(stream)), "mf_net_forward")
        return out

    def train_step(self, r, logk, target, lr, stream=None):
        self._fields("train_step", ("r", r), ("logk", logk), ("target", target))
        loss = C.c_float()
        check(lib.mf_net_train_step(self.h, _ptr(r), _ptr(logk), _ptr(target), float(lr), C.byref(loss),
                                    _stream(stream)), "mf_net_train_step")
        return loss.value

    def gradients(self, r, logk, target, stream=None):
        import numpy as np
        self._fields("gradients", ("r", r), ("logk", logk), ("target", target))
        g = np.empty(self.n_params, dtype=np.float32)
        loss = C.c_float()
        check(lib.mf_net_gradients(self.h, _ptr(r), _ptr(logk), _ptr(target), g.ctypes.data, C.byref(loss),
                                   _stream(stream)), "mf_net_gradients")
        return loss.value, g

    def close(self):
        if getattr(self, "h", None):
            check(lib.mf_net_destroy(self.h), "mf_net_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mf_operator_diagonal(h, diag, stream=None) -> None:
    check(lib.mf_operator_diagonal(h.h if isinstance(h, Mesh) else h, _ptr(diag), _stream(stream)), "mf_operator_diagonal")


def mf_training_pair(h, b, xs, xk, r32, e32, r64=None, e64=None, stream=None):
    """One training pair (see mf.h); returns (sum r~^2, sum e~^2)."""
    sums = (C.c_double * 2)()
    check(lib.mf_training_pair(h.h if isinstance(h, Mesh) else h, _ptr(b), _ptr(xs), _ptr(xk), _ptr(r64), _ptr(e64),
                               _ptr(r32), _ptr(e32), sums, _stream(stream)), "mf_training_pair")
    return float(sums[0]), float(sums[1])


def mf_kernel_launches() -> int:
    return int(lib.mf_kernel_launches())


def mf_last_error() -> str:
    return lib.mf_last_error().decode(errors="replace")


def mf_version() -> str:
    return lib.mf_version().decode()


# ----------------------------------------------------------------------------- handle owners ----

class Mesh:
    """Owner of an ``mf_mesh`` handle.  Arrays are torch tensors on the current CUDA device.
    ``element`` is "hex8" (Q1; ``cells`` None for a structured box of ``dims``), "tet4" (P1) or
    "hex27" (Q2); the last two need ``cells``."""

    def __init__(self, physics: str, coords, mat, dirichlet=None, cells=None, dims=None, stream=None,
                 element: str = "hex8"):
        self.physics = PHYSICS[physics]
        n_nodes = coords.shape[0]
        n_cells = cells.shape[0] if cells is not None else dims[0] * dims[1] * dims[2]
        nx, ny, nz = dims if (cells is None) else (0, 0, 0)
        self.dims = (nx, ny, nz)
        self._keep = (coords, mat, dirichlet, cells)
        if element == "hex8":
            self.h = mf_setup_mesh(self.physics, n_nodes, n_cells, coords, cells, nx, ny, nz, mat, dirichlet, stream)
        else:
            self.h = mf_setup_mesh_elem(ELEMENTS[element], self.physics, n_nodes, n_cells, coords, cells, mat,
                                        dirichlet, stream)
        self.info = mf_mesh_query(self.h)
        self._keep = None
        self.device = coords.device

    @classmethod
    def from_problem(cls, p, device="cuda", structured=True, stream=None):
        """Build from a ``paper_2308_09839_gb300.inputs.Problem``."""
        coords = torch.from_numpy(p.coords).to(device)
        mat = torch.from_numpy(p.mat).to(device).contiguous()
        dirichlet = torch.from_numpy(p.dirichlet).to(device)
        element = getattr(p, "element", "hex8")
        explicit = not structured or element != "hex8"
        cells = torch.from_numpy(p.cell_array()).to(device) if explicit else None
        return cls(p.physics, coords, mat, dirichlet, cells, (p.nx, p.ny, p.nz), stream, element=element)

    @property
    def n_dof(self) -> int:
        return self.info["n_dof"]

    def set_variant(self, variant: int) -> None:
        mf_set_apply_variant(self.h, variant)

    def apply(self, x, y=None, stream=None):
        n = self.info["n_dof"]
        _vec(x, n, (torch.float64, torch.float32), "Mesh.apply x")
        if y is None:
            y = torch.empty_like(x)
        _vec(y, n, (x.dtype,), "Mesh.apply y")
        if x.dtype == torch.float32:
            mf_apply_f32(self.h, x, y, stream)
        elif self.physics == MF_LAPLACE:
            mf_apply_laplace(self.h, x, y, stream)
        elif self.physics == MF_VECTOR_LAPLACE:
            mf_apply_vector_laplace(self.h, x, y, stream)
        else:
            mf_apply_elasticity(self.h, x, y, stream)
        return y

    def apply_multi(self, X, nrhs, Y=None, stream=None):
        n = self.info["n_dof"] * int(nrhs)
        _vec(X, n, (torch.float64,), "Mesh.apply_multi X")
        if Y is None:
            Y = torch.empty_like(X)
        _vec(Y, n, (torch.float64,), "Mesh.apply_multi Y")
        mf_apply_multi(self.h, nrhs, X, Y, stream)
        return Y

    def assemble_csr(self, stream=None) -> "Csr":
        return Csr(mf_assemble_csr(self.h, stream), self.device)

    def cg(self, b, x=None, stream=None, ok=(MF_OK, MF_NOT_CONVERGED), **kw):
        o = mf_solve_opts_default()
        csr = kw.pop("csr", None)
        net = kw.pop("net", None)
        if net is not None:
            o.net = net.h
            o.precond = MF_PC_LEARNED
        for k, v in kw.items():
            setattr(o, k, v)
        if csr is not None:
            o.csr = csr.h
            o.op = MF_OP_CSR
        n = self.info["n_dof"]
        _vec(b, n, (torch.float64,), "Mesh.cg b")
        if x is None:
            x = torch.empty_like(b)
        _vec(x, n, (torch.float64,), "Mesh.cg x")
        info = mf_cg_solve(self.h, o, b, x, stream, ok=ok)
        return x, info

    def cg_state(self, stream=None) -> bytes:
        return mf_cg_state_save(self.h, stream)

    def cg_resume(self, state: bytes, b, x=None, stream=None, ok=(MF_OK, MF_NOT_CONVERGED), **kw):
        o = mf_solve_opts_default()
        for k, v in kw.items():
            setattr(o, k, v)
        n = self.info["n_dof"]
        _vec(b, n, (torch.float64,), "Mesh.cg_resume b")
        if x is None:
            x = torch.empty_like(b)
        _vec(x, n, (torch.float64,), "Mesh.cg_resume x")
        info = mf_cg_resume(self.h, o, state, b, x, stream, ok=ok)
        return x, info

    def close(self):
        if getattr(self, "h", None):
            mf_destroy_mesh(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Csr:
    def __init__(self, h: int, device):
        self.h = h
        self.device = device
        self.info = mf_csr_query(h)

    def spmv(self, x, y=None, stream=None):
        n = self.info["n_rows"]
        _vec(x, n, (torch.float64,), "Csr.spmv x")
        if y is None:
            y = torch.empty_like(x)
        _vec(y, n, (torch.float64,), "Csr.spmv y")
        mf_spmv_csr(self.h, x, y, stream)
        return y

    def to_scipy(self):
        import scipy.sparse as sp
        q = self.info
        rp = torch.empty(q["n_rows"] + 1, dtype=torch.int64, device=self.device)
        cl = torch.empty(q["nnz"], dtype=torch.int32, device=self.device)
        vl = torch.empty(q["nnz"], dtype=torch.float64, device=self.device)
        mf_csr_export(self.h, rp, cl, vl)
        torch.cuda.synchronize()
        return sp.csr_matrix((vl.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(q["n_rows"], q["n_rows"]))

    def close(self):
        if getattr(self, "h", None):
            mf_destroy_csr(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
