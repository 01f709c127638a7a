"""C-ABI checks that need no GPU: the library builds for sm_103a, exports every function
that include/gbpic.h declares, and the Python mirror of pic_config has the C layout."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1604_07713_gb300 as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbpic.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"GBPIC_API\s+[\w\s\*]+?\b(pic_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    G.build()
    out = subprocess.run(["nm", "-D", "--defined-only", G.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(pic_\w+)", out))
    declared = _declared()
    assert len(declared) >= 18
    assert set(declared) <= exported, set(declared) - exported
    assert set(G.EXPORTED) == set(declared)
    L = C.CDLL(G.LIB_PATH)
    for name in declared:
        assert hasattr(L, name)


def test_config_struct_layout_matches_header(tmp_path):
    fields = [f[0] for f in G.PicConfig._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', 'int main(void){',
           'printf("%zu\\n", sizeof(pic_config));']
    for f in fields:
        src.append(f'printf("%zu\\n", offsetof(pic_config, {f}));')
    src.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", str(c), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == C.sizeof(G.PicConfig)
    for f, off in zip(fields, vals[1:]):
        assert getattr(G.PicConfig, f).offset == off, f


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(G, "_lib", None)
    monkeypatch.setattr(G, "LIB_PATH", "/nonexistent/libgbpic.so")
    with pytest.raises(RuntimeError):
        G.lib()


def test_bad_configuration_is_refused_before_any_device_call():
    from paper_1604_07713_gb300 import workloads as W
    G.build()
    for bad in (dict(precision=7), dict(n_species=3), dict(dt=0.0), dict(max_level=12), dict(mg_rel_tol=0.0),
                dict(shape=3), dict(shape=1, max_level=2)):
        cfg = W.base_config(**bad)
        with pytest.raises(G.PicError) as e:
            G.pic_create(cfg)
        assert e.value.status == G.PIC_EINVAL


def test_stability_limits_match_the_formulary_debye_length_and_plasma_frequency():
    """The explicit-PIC limits of §3 (h < ~3 lambda_D, omega_pe dt < 1) evaluated by the
    library's host function against the NRL plasma formulary's numerical forms
    lambda_D = 743 sqrt(T_e[eV] / n_e[cm^-3]) cm and omega_pe = 5.64e4 sqrt(n_e[cm^-3]) rad/s
    (three-digit constants: 1e-3 relative), for the capacitively coupled discharge's cells
    (h = 6.7 cm / 512, n = 1e15 m^-3, T_e = 2.5 eV, dt = 1 / (400 x 13.56 MHz)), and the
    warning thresholds on either side of the limits."""
    from paper_1604_07713_gb300 import workloads as W
    G.build()
    cfg, mesh, _ = W.ccp(nx=512, ny=16, ppc=1)
    h, n, te = mesh["h0"], 1e15, 2.5
    st, dx_ld, wdt = G.pic_stability_limits(cfg, n, n * h * h, te)
    lam = 743.0 * np.sqrt(te / (n * 1e-6)) * 1e-2
    wpe = 5.64e4 * np.sqrt(n * 1e-6)
    assert st == G.PIC_OK
    assert abs(dx_ld / (h / lam) - 1) < 1e-3 and abs(wdt / (wpe * cfg["dt"]) - 1) < 1e-3
    # densities 1 % above and below the one where h = 3 lambda_D
    n3 = n * 9.0 / (dx_ld / 1.0) ** 2
    assert G.pic_stability_limits(cfg, 0.0, 1.01 * n3 * h * h, te)[0] == G.PIC_WARN_STABILITY
    assert G.pic_stability_limits(cfg, 0.0, 0.99 * n3 * h * h, te)[0] == G.PIC_OK
    n1 = n / wdt ** 2                          # omega_pe dt = 1
    assert G.pic_stability_limits(cfg, 1.01 * n1, 0.0, te)[0] == G.PIC_WARN_STABILITY
    assert G.pic_stability_limits(cfg, 0.99 * n1, 0.0, te)[0] == G.PIC_OK
    # a cold population is never resolved; no electrons never warns
    st, dx_ld, _ = G.pic_stability_limits(cfg, n, n * h * h, 0.0)
    assert st == G.PIC_WARN_STABILITY and np.isinf(dx_ld)
    assert G.pic_stability_limits(cfg, 0.0, 0.0, 0.0)[0] == G.PIC_OK
    with pytest.raises(G.PicError):
        G.pic_stability_limits(cfg, -1.0, 0.0, te)
