"""Host-side checks of the C ABI: the library loads, exports every entry point that
include/lbpf.h declares, agrees with the header on the parameter struct layout,
and rejects bad arguments before it touches the GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2111_05960_gb300 import build as B
from paper_2111_05960_gb300 import lbpf as L
from paper_2111_05960_gb300 import workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbpf.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbpf_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lbpf_create" in names and "lbpf_step" in names and "lbpf_mass" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(L.exported_symbols()) | set(names)
    assert set(L.exported_symbols()) <= set(names)


def test_param_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    fields = [f[0] for f in L.lbpf_params._fields_]
    cfields = [("lambda" if f == "lambda_" else f) for f in fields]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbpf.h"', "int main(void){",
             'printf("%zu\\n", sizeof(lbpf_params));']
    lines += ['printf("%%zu\\n", offsetof(lbpf_params, %s));' % f for f in cfields]
    lines += ["return 0;}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert out[0] == ctypes.sizeof(L.lbpf_params)
    for f, off in zip(fields, out[1:]):
        assert getattr(L.lbpf_params, f).offset == off, f


def test_lattice_info_matches_oracle_and_paper(lib):
    for lat, code in ((L.LBPF_D2Q9, 2), (L.LBPF_D3Q19, 3), (L.LBPF_D2Q5, 5), (L.LBPF_D3Q7, 7)):
        e, w = L.lbpf_lattice_info(lat)
        eo, wo, _ = O.lattice_tables(code)
        assert np.array_equal(e, eo)
        assert np.array_equal(w, wo)
    with pytest.raises(L.LbpfError) as ei:
        L.lbpf_lattice_info(7)
    assert ei.value.status == L.LBPF_EINVAL


def test_default_params(lib):
    p = L.lbpf_default_params()
    assert (p.nx, p.ny, p.nz) == (64, 64, 1)
    assert p.precision == L.LBPF_FP64 and p.counter_term == 1 and p.a_at == -1.0
    assert (p.h_lattice, p.h_eq_alt, p.unequal_eps, p.eps_ratio) == (0, 0, 0, 1.0)


@pytest.mark.parametrize("mutate,msg", [
    (lambda p: setattr(p, "nx", 0), "grid sizes"),
    (lambda p: setattr(p, "nz", 4), "D2Q9 needs nz"),
    (lambda p: setattr(p, "lattice", 5), "unknown lattice"),
    (lambda p: setattr(p, "lattice", L.LBPF_D2Q5), "unknown lattice"),
    (lambda p: setattr(p, "h_lattice", 2), "h_lattice must be 0 or 1"),
    (lambda p: setattr(p, "h_eq_alt", -1), "h_eq_alt must be 0 or 1"),
    (lambda p: setattr(p, "unequal_eps", 3), "unequal_eps must be 0 or 1"),
    (lambda p: (setattr(p, "unequal_eps", 1), setattr(p, "eps_ratio", 0.0)), "eps_ratio"),
    (lambda p: setattr(p, "precision", 9), "unknown precision"),
    (lambda p: setattr(p, "tau_g", 0.0), "tau_g"),
    (lambda p: setattr(p, "W", -1.0), "W must be"),
    (lambda p: setattr(p, "D_s", -0.1), "diffusivities"),
    (lambda p: (p.bc.__setitem__(0, 1), setattr(p, "nx", 1)), "bounce-back axis"),
    (lambda p: p.bc.__setitem__(1, 3), "unknown boundary"),
    (lambda p: setattr(p, "lambda_", float("nan")), "non-finite"),
    (lambda p: setattr(p, "checkpoint_every", -1), "checkpoint_every"),
])
def test_create_rejects_bad_parameters_without_a_gpu(lib, mutate, msg):
    p = L.lbpf_default_params()
    mutate(p)
    n = max(p.nx, 1) * p.ny * max(p.nz, 1)
    a = np.zeros(n)
    with pytest.raises(L.LbpfError) as ei:
        L.lbpf_create(p, a, a, 0)
    assert ei.value.status == L.LBPF_EINVAL
    assert msg in str(ei.value)


def test_null_arguments(lib):
    p = L.lbpf_default_params()
    assert lib.lbpf_create(ctypes.byref(p), None, None, 0, None, None) == L.LBPF_EINVAL
    assert lib.lbpf_step(None, 1) == L.LBPF_EINVAL
    assert lib.lbpf_mass(None, None, None) == L.LBPF_EINVAL
    assert lib.lbpf_pull_path(None, None) == L.LBPF_EINVAL
    assert lib.lbpf_destroy(None) == L.LBPF_OK
    assert "NULL" in L.lbpf_last_error(None) or "ctx" in L.lbpf_last_error(None)


def test_params_from_workload_roundtrip(lib):
    m = WL.recipe(40, 30, D_l=0.1, D_s=0.0, W=2.0, counter_term=0, bc=(1, 0, 0))
    p = L.params_from(m, "fp32")
    assert (p.nx, p.ny, p.nz, p.lattice, p.precision) == (40, 30, 1, L.LBPF_D2Q9, L.LBPF_FP32)
    assert p.lambda_ == m.lam and p.a_at == m.a_at and p.anti_trapping == 1 and p.counter_term == 0


def test_create_batch_validates_on_the_host(lib):
    good = L.lbpf_default_params()
    a = np.zeros(64 * 64)
    bad = L.lbpf_default_params()
    bad.lattice, bad.nz = L.LBPF_D3Q19, 4
    b3 = np.zeros(64 * 64 * 4)
    with pytest.raises(L.LbpfError) as ei:
        L.lbpf_create_batch([good, bad], [a, b3], [a, b3])
    assert ei.value.status == L.LBPF_EUNSUPPORTED
    bad = L.lbpf_default_params()
    bad.mass_every = 1
    with pytest.raises(L.LbpfError) as ei:
        L.lbpf_create_batch([good, bad], [a, a], [a, a])
    assert ei.value.status == L.LBPF_EUNSUPPORTED
    bad = L.lbpf_default_params()
    bad.tau_h = -1.0
    with pytest.raises(L.LbpfError) as ei:
        L.lbpf_create_batch([good, bad], [a, a], [a, a])
    assert ei.value.status == L.LBPF_EINVAL and "instance 1" in str(ei.value)


def test_adjoint_arguments_are_checked_on_the_host(lib):
    out = np.zeros(len(L.ADJ_PARAM_NAMES))
    assert lib.lbpf_adjoint_step(None, None, None, None, None, 0,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == L.LBPF_EINVAL
    for prec in (L.LBPF_FP32_BF16DEV, L.LBPF_FP32_FP16DEV):
        p = L.lbpf_default_params()
        p.precision, p.checkpoint_every = prec, 10
        a = np.zeros(64 * 64)
        with pytest.raises(L.LbpfError) as ei:
            L.lbpf_create(p, a, a, 0)
        assert ei.value.status == L.LBPF_EUNSUPPORTED and "adjoint" in str(ei.value)
    good = L.lbpf_default_params()
    bad = L.lbpf_default_params()
    bad.checkpoint_every = 5
    a = np.zeros(64 * 64)
    with pytest.raises(L.LbpfError) as ei:
        L.lbpf_create_batch([good, bad], [a, a], [a, a])
    assert ei.value.status == L.LBPF_EUNSUPPORTED


def test_h_variants_rejected_where_not_built(lib):
    """The adjoint and the batches cover the main composition scheme only: h on
    the small lattice or with h^eq,alt is refused with EUNSUPPORTED before any
    device work."""
    a = np.zeros(64 * 64)
    for field in ("h_lattice", "h_eq_alt", "unequal_eps"):
        p = L.lbpf_default_params()
        setattr(p, field, 1)
        p.checkpoint_every = 10
        with pytest.raises(L.LbpfError) as ei:
            L.lbpf_create(p, a, a, 0)
        assert ei.value.status == L.LBPF_EUNSUPPORTED
        p.checkpoint_every = 0
        with pytest.raises(L.LbpfError) as ei:
            L.lbpf_create_batch([L.lbpf_default_params(), p], [a, a], [a, a])
        assert ei.value.status == L.LBPF_EUNSUPPORTED
        assert "instance" in str(ei.value) or "batches" in str(ei.value)


def test_params_from_carries_the_h_variants(lib):
    m = WL.recipe(40, 30, D_l=0.1, D_s=0.0, W=2.0)
    m.h_lattice, m.h_eq_alt = 1, 1
    p = L.params_from(m, "fp32")
    assert (p.h_lattice, p.h_eq_alt) == (1, 1)
