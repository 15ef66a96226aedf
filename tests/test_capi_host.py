"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every function include/gr.h declares, and arguments are
validated before any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_1905_08890_gb300 import gr

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gr.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gr_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_function():
    L = gr.lib()
    names = _declared()
    assert "gr_solve_constraints" in names and "gr_deposit" in names
    for name in names:
        assert hasattr(L, name), name


def test_default_opts():
    o = gr.make_opts()
    assert o.tol == 1e-10 and o.max_cycles == 50 and o.nu1 == 2 and o.nu2 == 2 and o.prec == 0


@pytest.mark.parametrize("n", [0, 2, 6, 12, 2048])
def test_bad_grid_size_rejected_without_gpu(n):
    h = ctypes.c_void_p()
    st = gr.lib().gr_create(n, 1.0, None, ctypes.byref(h))
    assert st == gr.GR_ERR_ARG and not h.value
    assert "power of two" in gr.gr_last_error()


def test_bad_box_and_null_arguments_rejected():
    h = ctypes.c_void_p()
    assert gr.lib().gr_create(8, -1.0, None, ctypes.byref(h)) == gr.GR_ERR_ARG
    assert gr.lib().gr_create(8, 1.0, None, None) == gr.GR_ERR_ARG
    o = gr.make_opts()
    assert gr.lib().gr_solve_constraints(None, None, None, ctypes.byref(o), None) == gr.GR_ERR_ARG
    assert gr.lib().gr_vcycle(None, 0, None, None, ctypes.byref(o), None) == gr.GR_ERR_ARG
    assert gr.lib().gr_residual(None, 0, None, None, ctypes.byref(o), None, None) == gr.GR_ERR_ARG
    assert gr.lib().gr_deposit(None, 0, None, None, 1.0, None) == gr.GR_ERR_ARG


def test_patch_deposit_rejects_null_context_and_bad_chains():
    p = gr.make_patches([{"n": 8, "origin": [0, 0, 0]}])
    assert gr.lib().gr_deposit_patches(None, 1, p, 0, None, None, 1.0) == gr.GR_ERR_ARG


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of gr_opts, gr_report and gr_patch have the C
    header's sizes and field offsets (compiled here with the host compiler)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    checks = {
        "gr_opts": ["tol", "max_cycles", "prec", "rho_hat", "fmg", "host_out", "npatch", "patch"],
        "gr_report": ["cycles", "res0", "seconds", "cell_updates", "prof_ms", "guess_rejected", "res_level"],
        "gr_patch": ["n", "origin", "src", "fld"],
    }
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "gr.h"', "int main(void) {"]
    for t, fields in checks.items():
        src.append(f'printf("{t} %zu\\n", sizeof({t}));')
        for f in fields:
            src.append(f'printf("{t}.{f} %zu\\n", offsetof({t}, {f}));')
    src.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(c), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for t, fields in checks.items():
        cls = getattr(gr, t)
        assert int(out[t]) == ctypes.sizeof(cls), t
        for f in fields:
            assert int(out[f"{t}.{f}"]) == getattr(cls, f).offset, (t, f)


def test_centred_chain_geometry():
    """gr.centred_chain: patch 1's block is centred on the cell (wrapping on
    the periodic base), each further patch sits in the middle of its parent,
    and every patch lies where the C chain check accepts it."""
    n0 = 512
    chain = gr.centred_chain(n0, (508, 3, 256), (128, 128))
    assert chain[0] == {"n": 128, "origin": [476, (3 - 32) % 512, 224]}
    assert chain[1] == {"n": 128, "origin": [32, 32, 32]}
    # the cell sits in the middle of both patches: base cell c covers patch-1 cells 2(c - o1) .. +1
    for d, c in enumerate((508, 3, 256)):
        i1 = 2 * ((c - chain[0]["origin"][d]) % n0)
        assert i1 == 64
        i2 = 2 * (i1 - chain[1]["origin"][d])
        assert i2 == 64
    for q, npar in zip(chain, (n0, 128)):
        for o in q["origin"]:
            if npar == n0:
                assert 0 <= o < n0 and q["n"] // 2 + 4 <= n0
            else:
                assert o >= 2 and o + q["n"] // 2 + 2 <= npar


def test_patch_options_marshalling():
    """make_opts(patches=...) fills npatch and a gr_patch array whose entries
    carry n, origin and NULL arrays where none are given."""
    chain = [{"n": 16, "origin": [1, 2, 3]}, {"n": 8, "origin": [4, 5, 6]}]
    o = gr.make_opts(patches=chain)
    assert o.npatch == 2
    assert o.patch[0].n == 16 and list(o.patch[0].origin) == [1, 2, 3]
    assert o.patch[1].n == 8 and list(o.patch[1].origin) == [4, 5, 6]
    assert not o.patch[0].src.s0 and not o.patch[1].fld.psi
    assert gr.make_opts().npatch == 0 and not gr.make_opts().patch


def test_particle_entry_points_reject_bad_arguments_without_gpu():
    L = gr.lib()
    f = gr.gr_fields()
    assert L.gr_particle_update(None, 0, None, None, ctypes.byref(f), 0.1, 7) == gr.GR_ERR_ARG
    assert L.gr_kick(None, 0, None, None, ctypes.byref(f), 0.1, gr.GR_DRIFT) == gr.GR_ERR_ARG
    assert "flags" in gr.gr_last_error()
    assert L.gr_drift(None, 0, None, None, ctypes.byref(f), 0.1) == gr.GR_ERR_ARG
    assert L.gr_deposit_metric(None, 0, None, None, 1.0, None, None) == gr.GR_ERR_ARG


def test_code_unit_entry_point_rejects_bad_arguments_without_gpu():
    o = gr.make_opts()
    cm = gr.gr_cosmology(1.0, 1.0, 0.0, 1.0 / 3.0)
    assert gr.lib().gr_solve_code_units(None, ctypes.byref(cm), None, None, ctypes.byref(o), None) == gr.GR_ERR_ARG


def test_fma_rate_rejects_bad_arguments_without_gpu():
    L = gr.lib()
    out = ctypes.c_double(-1.0)
    assert L.gr_fma_rate(1, 0, None, ctypes.byref(out)) == gr.GR_ERR_ARG
    assert L.gr_fma_rate(0, (1 << 32) + 1, None, ctypes.byref(out)) == gr.GR_ERR_ARG
    assert L.gr_fma_rate(1, 100, None, None) == gr.GR_ERR_ARG
