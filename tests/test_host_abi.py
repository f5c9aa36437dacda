"""Host-side checks of the C ABI (CPU only, no CUDA call is made).

* libkb.so loads and exports every function include/kb.h declares.
* kb_graph_create rejects malformed Laplacians before touching the GPU.
* The host coefficient math of the Chebyshev steps agrees with the oracle.
"""
import os
import re

import numpy as np
import pytest

import synth
from oracle import dense, krylov

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kb():
    from paper_2301_06384_gb300 import kb as _kb
    if not os.path.exists(_kb.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    _kb.lib()
    return _kb


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(kb_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol(kb):
    names = _declared_functions()
    assert {"kb_graph_create", "kb_krylov_apply", "kb_krylov_apply_host"} <= names
    L = kb.lib()
    for name in sorted(names):
        assert hasattr(L, name), name


def test_version_and_status_strings(kb):
    L = kb.lib()
    assert L.kb_version() >= 10000
    for code in kb.STATUS:
        assert L.kb_status_string(code)


def _expect(kb, code, *args, **kw):
    with pytest.raises(kb.KbError) as ei:
        kb.Graph(*args, **kw)
    assert ei.value.code == code, str(ei.value)


def test_csr_validation_rejects_malformed_input(kb):
    g = synth.path_graph(6)
    # unsorted columns
    col = g.col.copy(); col[[0, 1]] = col[[1, 0]]
    _expect(kb, -2, g.rowptr, col, g.val)
    # out of range column
    col = g.col.copy(); col[-1] = 99
    _expect(kb, -2, g.rowptr, col, g.val)
    # non-symmetric value
    val = g.val.copy(); val[1] = -2.0
    _expect(kb, -2, g.rowptr, g.col, val)
    # positive off-diagonal
    val = g.val.copy(); val[1] = 1.0
    idx = np.where((g.col == 0) & (np.repeat(np.arange(6), np.diff(g.rowptr)) == 1))[0]
    val[idx] = 1.0
    _expect(kb, -2, g.rowptr, g.col, val)
    # non-monotone rowptr
    rp = g.rowptr.copy(); rp[2] = rp[3] + 1
    _expect(kb, -2, rp, g.col, g.val)
    # bad n
    _expect(kb, -1, np.zeros(1, np.int32), np.zeros(0, np.int32), None)
    # non-symmetric pattern (drop one off-diagonal entry of row 0)
    rp = g.rowptr.copy(); rp[1:] -= 1
    col = np.delete(g.col, 1); val = np.delete(g.val, 1)
    _expect(kb, -2, rp, col, val)


@pytest.mark.parametrize("m", [1, 2, 7, 30])
@pytest.mark.parametrize("phi,kw", [("exp", dict(t=0.5)), ("exp", dict(t=2.0)),
                                    ("spline", dict(eps=0.01, s=2.0)), ("spline", dict(eps=0.05, s=1.5))])
@pytest.mark.parametrize("sq", [False, True])
def test_lobatto_coefficients_match_oracle(kb, m, phi, kw, sq):
    lam = 46.0
    c = kb.kb_cheb_lobatto_coeffs(phi, kb.make_params(**kw), m, lam, sqrt_phi=sq)
    f = (dense.sqrt_phi_function if sq else dense.phi_function)(phi, **kw)
    ref = krylov.cheb_coefficients(f, m, lam)
    assert np.max(np.abs(c - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("t,lam", [(0.5, 60.0), (2.0, 60.0), (0.01, 8.0), (5.0, 200.0), (-0.2, 10.0)])
def test_exp_series_reproduces_exponential(kb, t, lam):
    d = kb.kb_exp_series_coeffs(t, lam)
    x = np.cos(np.linspace(0, np.pi, 257))
    T = np.cos(np.outer(np.arccos(x), np.arange(d.size)))
    lmb = 0.5 * lam * (1 - x)
    ref = np.exp(-t * lmb)
    assert np.max(np.abs(T @ d - ref) / np.maximum(ref, 1e-300 + np.abs(ref).max())) < 1e-14


@pytest.mark.parametrize("s", [0.5, 0.25, 0.9, 1.5, 2.3])
@pytest.mark.parametrize("eps,lam", [(0.1, 20.0), (0.01, 60.0), (1e-3, 3000.0)])
def test_spline_quadrature_reproduces_the_fractional_power(kb, eps, s, lam):
    # (eps + lambda)^{-s} = (eps + lambda)^{-floor(s)} sum_k W_k / (sigma_k + lambda) on
    # [0, Lambda], checked against pow at points the rule's own grid does not use
    sh, w, s_int = kb.kb_spline_quadrature(eps, s, lam)
    assert s_int == int(np.floor(s)) and np.all(sh > eps) and np.all(w > 0)
    rng = np.random.default_rng(5)
    lmb = np.concatenate([lam * rng.random(500), eps * np.expm1(np.log1p(lam / eps) * rng.random(500))])
    approx = (eps + lmb) ** (-s_int) * (w[None, :] / (sh[None, :] + lmb[:, None])).sum(axis=1)
    ref = (eps + lmb) ** (-s)
    assert np.max(np.abs(approx - ref) / ref) < 1e-13
    assert sh.size <= 240


@pytest.mark.parametrize("alpha", [0.5, 0.2, 0.85])
def test_spline_quadrature_nodes_are_gauss_jacobi(kb, alpha):
    # the rule's nodes and weights, mapped back to [-1, 1] (t = c u^3, u = (1-x)/(1+x)), are
    # the Gauss-Jacobi rule of the weight (1-x)^{3(1-alpha)-1} (1+x)^{3 alpha-1} (library
    # reference: scipy.special.roots_jacobi)
    from scipy.special import roots_jacobi
    eps, lam = 0.02, 50.0
    sh, w, _ = kb.kb_spline_quadrature(eps, 1.0 + alpha, lam)
    c = np.sqrt(eps * (eps + lam))
    u = np.cbrt((sh - eps) / c)
    x = (1 - u) / (1 + u)
    pre = c ** (1 - alpha) * 6 * np.sin(np.pi * alpha) / np.pi
    wj = w * (1 + x) ** 3 / pre
    order = np.argsort(x)
    xr, wr = roots_jacobi(sh.size, 3 * (1 - alpha) - 1, 3 * alpha - 1)
    # mapping a shift back to x loses digits where sigma - eps << eps (x near 1): compare
    # the nodes where the map is well conditioned, the weights everywhere
    ok = ((sh - eps) / eps > 1e-4)[order]
    assert ok.sum() >= 0.9 * sh.size
    assert np.max(np.abs(x[order] - xr)[ok]) < 1e-12
    assert np.max(np.abs(wj[order] - wr) / wr.max()) < 1e-10


def test_spline_quadrature_integer_s_and_errors(kb):
    sh, w, s_int = kb.kb_spline_quadrature(0.1, 3.0, 10.0)
    assert sh.size == 0 and s_int == 3
    for args in [(0.0, 1.5, 10.0), (0.1, -1.0, 10.0), (0.1, 1.5, 0.0), (float("inf"), 1.5, 1.0)]:
        with pytest.raises(kb.KbError) as ei:
            kb.kb_spline_quadrature(*args)
        assert ei.value.code == -1


def test_binding_struct_layouts_match_the_header(kb, tmp_path):
    # the ctypes mirrors of the ABI structs have the C sizes and field offsets (a plain C
    # program compiled against include/kb.h prints them; gcc, no CUDA)
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"kb_params": kb.kb_params, "kb_info": kb.kb_info,
               "kb_server_config": kb.kb_server_config}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "kb.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            sname, key, val = line.split()
            got[(sname, key)] = int(val)
    for sname, cls in structs.items():
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)
