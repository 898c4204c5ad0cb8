"""The C ABI library loads and exports every call that include/lbib.h
declares; host-side argument checks run without a GPU."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1808_01448_gb300 import build, lbib
    build.build()
    return lbib


def declared(path):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbib_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared(os.path.join(ROOT, "include", "lbib.h"))
    for n in ("lbib_create", "lbib_add_particle", "lbib_set_receptors", "lbib_step",
              "lbib_read_state", "lbib_destroy", "lbib_batch_step", "lbib_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names += declared(os.path.join(ROOT, "include", h))
    lib = L.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\sT\s(lbib_\w+)", out))
    assert set(names) <= exported


def test_version_and_error_text(L):
    assert "sm_103a" in L.version()


@pytest.mark.parametrize("bad", [dict(nx=4), dict(ny=2), dict(tau=0.5), dict(tau=-1.0),
                                 dict(wall_bottom="periodic"), dict(storage=9),
                                 dict(kBT=0.0), dict(eps_min=0.0)])
def test_invalid_configs_are_rejected_before_any_device_call(L, bad):
    with pytest.raises(L.LbibError) as e:
        L.Sim(**bad)
    assert e.value.status == "E_ARG"
