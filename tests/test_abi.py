"""The C-ABI library loads and exports every function ``include/mf.h`` declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2308_09839_gb300", "libmf.so")


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:mf_status|void|int64_t|const char \*)\s*\*?\s*(mf_\w+)\s*\(", txt, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2308_09839_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for required in ("mf_setup_mesh", "mf_apply_laplace", "mf_apply_elasticity", "mf_spmv_csr", "mf_cg_solve",
                     "mf_assemble_csr", "mf_last_error"):
        assert required in names


def test_every_declaration_is_documented():
    """Each function of the boundary has a comment: directly above its declaration, or in the block
    comment of its group that names it."""
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        lines = open(os.path.join(ROOT, "include", fn)).read().splitlines()
        decl = re.compile(r"^\s*(?:mf_status|void|int64_t|size_t|const char \*)\s*\*?\s*(mf_\w+)\s*\(")
        comments = []
        for i, line in enumerate(lines):
            m = decl.match(line)
            if not m:
                continue
            above = lines[i - 1].strip()
            block = "\n".join(ln for ln in lines[max(0, i - 80):i] if ln.lstrip().startswith(("/*", "*")))
            if not (above.endswith("*/") or m.group(1) in block):
                comments.append(m.group(1))
        assert not comments, (fn, comments)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(lib):
    from paper_2308_09839_gb300 import mf
    assert set(declared_functions()) <= set(mf.EXPORTED)


def test_library_is_built_for_sm_103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", LIB], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_host_only_calls(lib):
    """Calls that need no device: version string and argument validation paths."""
    from paper_2308_09839_gb300 import mf
    assert mf.mf_version().startswith("mf-gb300")
    o = mf.mf_solve_opts_default()
    assert o.rtol == 1e-8 and o.check_every == 32 and o.use_graph == 1
    # a null mesh handle is rejected before any CUDA call
    assert mf.lib.mf_apply_laplace(None, None, None, None) == mf.MF_ERR_ARG
    assert "null" in mf.mf_last_error()
    info = {}
    assert mf.lib.mf_mesh_query(None, None, None, None, None, None, None) == mf.MF_ERR_ARG


def test_setup_refuses_meshes_beyond_32_bit_indices(lib):
    """3 N and npe E must fit int32 (the kernels' index type): the setup refuses larger meshes with
    MF_ERR_ARG before it touches a pointer or the device (the dummy pointers are never read)."""
    import ctypes as C
    from paper_2308_09839_gb300 import mf
    fake = C.c_void_p(16)
    out = C.c_void_p()
    big_nodes = (2 ** 31) // 3 + 1
    assert mf.lib.mf_setup_mesh(mf.MF_LAPLACE, big_nodes, 1000, fake, fake, 0, 0, 0, fake, None, None,
                                C.byref(out)) == mf.MF_ERR_ARG
    assert "3 n_nodes must fit int32" in mf.mf_last_error() and not out.value
    big_cells = (2 ** 31) // 8 + 1
    assert mf.lib.mf_setup_mesh(mf.MF_LAPLACE, 1000, big_cells, fake, fake, 0, 0, 0, fake, None, None,
                                C.byref(out)) == mf.MF_ERR_ARG
    assert "connectivity" in mf.mf_last_error() and not out.value
    # 27-node cells reach the limit 27/8 times sooner
    q2_cells = (2 ** 31) // 27 + 1
    assert mf.lib.mf_setup_mesh_elem(mf.MF_ELEM_HEX27, mf.MF_LAPLACE, 1000, q2_cells, fake, fake, fake, None, None,
                                     C.byref(out)) == mf.MF_ERR_ARG
    assert "27 nodes" in mf.mf_last_error() and not out.value


def test_release_build_reports_no_index_checks(lib):
    """mf_debug_status in the release library: checks compiled out, no device touched."""
    from paper_2308_09839_gb300 import mf
    if os.environ.get("MF_LIB"):
        pytest.skip("another build of the library is loaded")
    assert mf.mf_debug_status() == (0, False)


C_PROGRAM = r"""
#include "mf.h"
#include <stdio.h>
int main(void) {
  mf_solve_opts o;
  uint32_t bits = 1;
  int32_t enabled = 1;
  mf_status s;
  mf_solve_opts_default(&o);
  s = mf_debug_status(&bits, &enabled);
  printf("%s %g\n", mf_version(), o.rtol);
  /* argument checks happen before any device call */
  if (mf_apply_laplace(NULL, NULL, NULL, NULL) != MF_ERR_ARG) return 2;
  if (mf_spmv_csr(NULL, NULL, NULL, NULL) != MF_ERR_ARG) return 3;
  return s != MF_OK || bits != 0u || enabled != 0;
}
"""


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/mf.h compiles as strict C99 (no C++ in the boundary) and a C program links libmf.so
    and runs its host-only calls."""
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("gcc unavailable")
    if os.environ.get("MF_LIB"):
        pytest.skip("another build of the library is loaded")
    src = tmp_path / "use_mf.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_mf"
    pkg = os.path.dirname(LIB)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", pkg, "-l:libmf.so", f"-Wl,-rpath,{pkg}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    assert run.stdout.startswith("mf-gb300")


def test_ctypes_structs_and_constants_match_the_header(lib, tmp_path):
    """The binding's view of the boundary equals the C compiler's: every field offset and the size of
    mf_solve_opts and mf_solve_info, and the value of every MF_* integer constant mf.py defines (a
    name the header lacks fails to compile)."""
    import ctypes
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("gcc unavailable")
    from paper_2308_09839_gb300 import mf
    lines = ['#include "mf.h"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    expect = []
    for st in (mf.mf_solve_opts, mf.mf_solve_info):
        name = st.__name__
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        expect.append(ctypes.sizeof(st))
        for field, _ in st._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {field}));')
            expect.append(getattr(st, field).offset)
    consts = sorted(k for k, v in vars(mf).items() if k.startswith("MF_") and isinstance(v, int))
    assert len(consts) > 20
    for k in consts:
        lines.append(f'  printf("%lld\\n", (long long)({k}));')
        expect.append(getattr(mf, k))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == expect


def test_vector_arguments_are_checked_before_the_library(lib):
    """Mesh and Csr methods refuse vectors that the kernels would read or write out of bounds (another
    dtype, too few elements, y of another precision than x) before any call into the library; valid
    host tensors get past these checks and stop at the CUDA-tensor check."""
    import torch
    from paper_2308_09839_gb300 import mf
    m = mf.Mesh.__new__(mf.Mesh)
    m.h, m.physics, m.info = None, mf.MF_ELASTICITY, {"n_dof": 24}
    f64, f32 = torch.float64, torch.float32
    cases = [
        (lambda: m.apply(torch.zeros(24, dtype=torch.float16)), "dtype"),
        (lambda: m.apply(torch.zeros(23, dtype=f64)), "23 elements; 24 needed"),
        (lambda: m.apply(torch.zeros(24, dtype=f64), torch.zeros(24, dtype=f32)), "Mesh.apply y: dtype"),
        (lambda: m.apply_multi(torch.zeros(24 * 3 - 1, dtype=f64), 3), "71 elements; 72 needed"),
        (lambda: m.cg(torch.zeros(24, dtype=f32)), "Mesh.cg b: dtype"),
        (lambda: m.cg(torch.zeros(24, dtype=f64), torch.zeros(20, dtype=f64)), "Mesh.cg x: 20 elements"),
        (lambda: m.cg_resume(b"", torch.zeros(10, dtype=f64)), "Mesh.cg_resume b: 10 elements"),
        (lambda: m.apply(torch.zeros(24, dtype=f64)), "expected a CUDA tensor"),
        (lambda: m.apply(torch.zeros(24, dtype=f32)), "expected a CUDA tensor"),
        (lambda: m.apply_multi(torch.zeros(72, dtype=f64), 3), "expected a CUDA tensor"),
        (lambda: m.cg(torch.zeros(24, dtype=f64)), "expected a CUDA tensor"),
    ]
    a = mf.Csr.__new__(mf.Csr)
    a.h, a.info = None, {"n_rows": 24}
    cases += [(lambda: a.spmv(torch.zeros(24, dtype=f32)), "Csr.spmv x: dtype"),
              (lambda: a.spmv(torch.zeros(24, dtype=f64), torch.zeros(2, dtype=f64)), "Csr.spmv y: 2 elements"),
              (lambda: a.spmv(torch.zeros(24, dtype=f64)), "expected a CUDA tensor")]
    nt = mf.Net.__new__(mf.Net)
    nt.h, nt.dims = None, (5, 5, 9)
    v = torch.zeros(225, dtype=f32)
    cases += [(lambda: nt.forward(torch.zeros(225, dtype=torch.float16), v), "Net.forward r: dtype"),
              (lambda: nt.forward(v, torch.zeros(224, dtype=f32)), "Net.forward logk: 224 elements"),
              (lambda: nt.train_step(v, v, torch.zeros(225, dtype=f64), 1e-3), "Net.train_step target: dtype"),
              (lambda: nt.gradients(v, v, v[:100]), "Net.gradients target: 100 elements"),
              (lambda: nt.forward(v, v), "expected a CUDA tensor"),
              (lambda: nt.train_step(v, v, v, 1e-3), "expected a CUDA tensor")]
    for call, msg in cases:
        with pytest.raises(ValueError, match=msg):
            call()
