"""The C-ABI library builds, loads without a GPU, and exports every function
include/qrdm.h declares; argument checks run on the host (no compute)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qrdm.h")


def declared_functions() -> list[str]:
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(qrdm_[a-z_0-9]+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_03138_gb300 import _binding

    return _binding.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    assert "qrdm_factor" in names and "qrdm_workspace_size" in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2106_03138_gb300 import _binding

    so = _binding.lib_path()
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(_binding.EXPORTS) == set(declared_functions())


STRUCTS = ("qrdm_opts", "qrdm_policy", "qrdm_info", "qrdm_profile", "qrdm_step_record", "qrdm_batch_matrix",
           "qrdm_batch_tuning")


def c_layouts(tmp_path) -> dict:
    """sizeof and offsetof of every field, as a C compiler lays out the
    header's structs (gcc on the header alone)."""
    from paper_2106_03138_gb300 import _binding

    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for st in STRUCTS:
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f, _ in getattr(_binding, st)._fields_:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    res = {}
    for line in out.splitlines():
        st, f, v = line.split()
        res[(st, f)] = int(v)
    return res


def test_struct_layouts(tmp_path):
    """The ctypes structs of the binding match the header field by field."""
    from paper_2106_03138_gb300 import _binding

    lay = c_layouts(tmp_path)
    for st in STRUCTS:
        cls = getattr(_binding, st)
        assert ctypes.sizeof(cls) == lay[(st, "size")], st
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == lay[(st, f)], (st, f)


def test_workspace_size_and_argument_checks(lib):
    from paper_2106_03138_gb300 import _binding as b

    n1 = b.qrdm_workspace_size(256, 256, 32)
    n2 = b.qrdm_workspace_size(4096, 4096, 64)
    assert 0 < n1 < n2
    # the shapes the header promises to the fixed scratch of qrdm_factor_noalloc
    scratch = 32 << 20
    assert b.qrdm_workspace_size(4096, 4096, 32) <= scratch
    assert b.qrdm_workspace_size(2048, 2048, 64) <= scratch
    # blocks of at most 64 columns also hold the tensor-core forms' operand
    # images (512 B per padded row of V twice and per padded column of W)
    img = (2 * (4096 + 256) + (4096 + 256)) * 512
    assert b.qrdm_workspace_size(4096, 4096, 64) >= img
    with pytest.raises(ValueError):
        b.qrdm_workspace_size(-1, 4, 4)
    with pytest.raises(ValueError):
        b.qrdm_workspace_size(4, 4, 0)
    with pytest.raises(ValueError):
        b.qrdm_workspace_size(4, 4, 129)
    # invalid arguments are rejected before any CUDA call (LAPACK-style -i)
    fake = 1 << 20  # never dereferenced
    rc, _ = b.qrdm_factor(fake, -1, 4, 4, 0.5, 0.5, 4, fake, fake, None, fake, 1 << 30, 0)
    assert rc == -1
    rc, _ = b.qrdm_factor(fake, 4, 4, 3, 0.5, 0.5, 4, fake, fake, None, fake, 1 << 30, 0)
    assert rc == -4
    rc, _ = b.qrdm_factor(fake, 4, 4, 4, 0.0, 0.5, 4, fake, fake, None, fake, 1 << 30, 0)
    assert rc == -5
    rc, _ = b.qrdm_factor(fake, 4, 4, 4, 0.5, 1.5, 4, fake, fake, None, fake, 1 << 30, 0)
    assert rc == -6
    rc, _ = b.qrdm_factor(fake, 4, 4, 4, 0.5, 0.5, 0, fake, fake, None, fake, 1 << 30, 0)
    assert rc == -7
    rc, _ = b.qrdm_factor(fake, 4, 4, 4, 0.5, 0.5, 4, 0, fake, None, fake, 1 << 30, 0)
    assert rc == -8
    o = b.qrdm_opts()
    o.eps1_mode = 7
    rc, _ = b.qrdm_factor(fake, 4, 4, 4, 0.5, 0.5, 4, fake, fake, o, fake, 1 << 30, 0)
    assert rc == -11
    o = b.qrdm_opts()
    for bad in (5, -1):
        o.precision = bad
        rc, _ = b.qrdm_factor(fake, 4, 4, 4, 0.5, 0.5, 4, fake, fake, o, fake, 1 << 30, 0)
        assert rc == -11
    o.precision = 3  # the tensor-core forms take blocks of at most 64
    rc, _ = b.qrdm_factor(fake, 4, 4, 4, 0.5, 0.5, 65, fake, fake, o, fake, 1 << 30, 0)
    assert rc == b.QRDM_ERR_UNSUPPORTED
    # checked, wait limit and test hook values
    for field, bad in (("checked", 2), ("checked", -1), ("wait_limit_us", -5), ("test_fault", 4),
                       ("test_fault", -1), ("test_fault", 2), ("test_fault", 3)):
        o = b.qrdm_opts()
        setattr(o, field, bad)  # hook 2 needs checked = 1, hook 3 a tensor-core precision
        rc, _ = b.qrdm_factor(fake, 4, 4, 4, 0.5, 0.5, 4, fake, fake, o, fake, 1 << 30, 0)
        assert rc == -11, (field, bad)
    # the same checks apply to an empty matrix (nothing to factor)
    o = b.qrdm_opts()
    o.precision = 9
    rc, _ = b.qrdm_factor(0, 0, 4, 1, 0.5, 0.5, 4, 0, fake, o, 0, 0, 0)
    assert rc == -11
    rc, _ = b.qrdm_factor_noalloc(0, 0, 4, 1, 0.5, 0.5, 4, 0, fake, o, 0)
    assert rc == -11
    o.precision = 2
    rc, _ = b.qrdm_factor_noalloc(0, 4, 0, 4, 0.5, 0.5, 65, 0, 0, o, 0)
    assert rc == b.QRDM_ERR_UNSUPPORTED
    assert b.qrdm_strerror(2).startswith("the matrix")
    assert b.qrdm_strerror(b.QRDM_ERR_TIMEOUT).startswith("a bounded")
    assert b.qrdm_strerror(b.QRDM_ERR_CHECKED).startswith("a checked")
    assert lib.qrdm_version() >= 200


def test_batched_struct_layouts():
    from paper_2106_03138_gb300 import _binding

    assert ctypes.sizeof(_binding.qrdm_batch_matrix) == 96
    assert ctypes.sizeof(_binding.qrdm_batch_tuning) == 16


def test_batched_argument_checks(lib):
    from paper_2106_03138_gb300 import _binding as b

    fake = 1 << 20  # never dereferenced
    good = b.qrdm_batch_matrix(fake, 8, 4, 8, fake, fake, None, None, 0, None, None, 0)
    # invalid arguments are rejected before any CUDA call
    h = ctypes.c_void_p(0)
    arr = (b.qrdm_batch_matrix * 1)(good)
    assert lib.qrdm_batch_plan_create(-1, arr, 4, ctypes.byref(h)) == -1
    assert lib.qrdm_batch_plan_create(1, None, 4, ctypes.byref(h)) == -2
    assert lib.qrdm_batch_plan_create(1, arr, 0, ctypes.byref(h)) == -3
    assert lib.qrdm_batch_plan_create(1, arr, 129, ctypes.byref(h)) == -3
    assert lib.qrdm_batch_plan_create(1, arr, 4, None) == -4
    for bad in (b.qrdm_batch_matrix(fake, -1, 4, 8, fake, fake, None, None, 0),       # m < 0
                b.qrdm_batch_matrix(fake, 8, 4, 7, fake, fake, None, None, 0),        # lda < m
                b.qrdm_batch_matrix(None, 8, 4, 8, fake, fake, None, None, 0),        # no A
                b.qrdm_batch_matrix(fake, 8, 4, 8, None, fake, None, None, 0),        # no htau
                b.qrdm_batch_matrix(fake, 8, 4, 8, fake, None, None, None, 0),        # no perm
                b.qrdm_batch_matrix(fake, 8, 4, 8, fake, fake, None, None, 3, None, None, 0),  # trace_cap, no trace
                b.qrdm_batch_matrix(fake, 8, 4, 8, fake, fake, None, None, 0, None, None, -1)):  # log_cap < 0
        arr2 = (b.qrdm_batch_matrix * 2)(good, bad)
        assert lib.qrdm_batch_plan_create(2, arr2, 4, ctypes.byref(h)) == -2
    # a NULL plan is refused by every call; destroying it is a no-op
    out = ctypes.c_size_t(0)
    assert lib.qrdm_batch_workspace_size(None, ctypes.byref(out)) == -1
    assert lib.qrdm_batch_bind(None, fake, 1 << 20, None) == -1
    assert lib.qrdm_factor_batched(None, 0.5, 0.5, None, None) == -1
    assert lib.qrdm_factor_batched_graph(None, 0.5, 0.5, None, None) == -1
    assert lib.qrdm_batch_results(None, None, None, None, None, None) == -1
    t = b.qrdm_batch_tuning()
    assert lib.qrdm_batch_get_tuning(None, ctypes.byref(t)) == -1
    assert lib.qrdm_batch_set_tuning(None, ctypes.byref(t)) == -1
    assert lib.qrdm_batch_autotune(None, 0.5, 0.5, None, None, None, None) == -1
    lib.qrdm_batch_plan_destroy(None)


def test_policy_and_mlp_argument_checks(lib):
    from paper_2106_03138_gb300 import _binding as b

    fake = 1 << 20  # never dereferenced
    pol = b.qrdm_policy(None, None, None, 0, 0.1, 1.0, 0.5, 1.0, 0.05)
    for field, bad in (("tau_lo", 0.0), ("tau_hi", 1.5), ("delta_lo", -0.1), ("rho_min", -1.0), ("log_cap", -3)):
        p = b.qrdm_policy.from_buffer_copy(pol)
        setattr(p, field, bad)
        o = b.qrdm_opts()
        o.policy = ctypes.pointer(p)
        rc, _ = b.qrdm_factor(fake, 4, 4, 4, 0.5, 0.5, 4, fake, fake, o, fake, 1 << 30, 0)
        assert rc == -11, field
    assert b.qrdm_mlp_workspace_size(64) > 0
    with pytest.raises(ValueError):
        b.qrdm_mlp_workspace_size(0)
    assert lib.qrdm_mlp_init(None, fake, 1, None) == -1
    assert lib.qrdm_mlp_init(fake, None, 1, None) == -2
    assert lib.qrdm_mlp_forward(fake, fake, 0, fake, fake, 1 << 30, None) == -3
    assert lib.qrdm_mlp_forward(fake, fake, 4, fake, fake, 16, None) == b.QRDM_ERR_WORKSPACE
    assert lib.qrdm_mlp_loss_grad(fake, fake, None, 4, fake, fake, fake, 1 << 30, None) == -3
    assert lib.qrdm_mlp_adam_step(fake, fake, fake, fake, fake, 0, 1e-3, 0.9, 0.999, 1e-8, 0.0, None) == -6
    assert lib.qrdm_mlp_adam_step(fake, fake, fake, fake, fake, 1, 1e-3, 1.0, 0.999, 1e-8, 0.0, None) == -8
    assert lib.qrdm_mlp_train(fake, fake, fake, fake, fake, 0, 4, 1, 1e-3, 0.0, 1, None, fake, 1 << 30, None) == -6
    assert lib.qrdm_mlp_train(fake, fake, fake, fake, fake, 10, 4, 1, -1.0, 0.0, 1, None, fake, 1 << 30, None) == -9


def test_the_library_path_has_no_fallback(monkeypatch):
    """The product path fails loudly when libqrdm.so is missing, and no
    module of the package imports the CPU oracle (which is test
    infrastructure only): there is no CPU fallback to land on."""
    import ast
    import glob

    from paper_2106_03138_gb300 import _binding, build as _build

    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_build, "LIB", os.path.join(os.path.dirname(_build.LIB), "no_such_libqrdm.so"))
    with pytest.raises(RuntimeError):
        _binding.load(build_if_missing=False)
    pkg = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2106_03138_gb300")
    for f in glob.glob(os.path.join(pkg, "*.py")):
        tree = ast.parse(open(f).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            else:
                continue
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), (f, mods)


def test_the_oracle_shares_no_code_with_the_gpu_path():
    """The oracle imports nothing from the package and includes none of its
    headers; the CUDA sources include nothing from the oracle."""
    import ast
    import glob

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for f in glob.glob(os.path.join(root, "oracle", "*.py")):
        for node in ast.walk(ast.parse(open(f).read())):
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            else:
                continue
            assert not any(m.startswith("paper_2106_03138_gb300") for m in mods), (f, mods)
    for f in glob.glob(os.path.join(root, "oracle", "*.c")):
        incs = re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(f).read())
        assert all("/" not in i and not i.startswith("qrdm") for i in incs), (f, incs)
    for f in glob.glob(os.path.join(root, "paper_2106_03138_gb300", "csrc", "*.c*")):
        incs = re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(f).read())
        assert not any("oracle" in i or i.startswith("oq_") for i in incs), (f, incs)
