"""Pins of the oracle's subsystem step (diagonalise + truncate) against facts the
paper and the mathematics fix, independent of the oracle's own formulas."""
import json
import os

import numpy as np
import pytest

from oracle.subsystems import (build_mode, mathieu_transmon_levels, transmon, fluxonium,
                               diagonalise, mode_derivatives, gauge_fix)

GHZ = 2.0 * np.pi
HERE = os.path.dirname(os.path.abspath(__file__))


def test_transmon_matches_mathieu_characteristic_values():
    # n_g = 0 transmon levels are E_C * {a0, b2, a2, b4}(q = -E_J/2E_C): a closed
    # form from scipy's Mathieu routines, not from the charge-basis matrix.
    for ej, ec in [(15.0, 0.3), (20.0, 0.25), (25.0, 0.2)]:
        ej, ec = ej * GHZ, ec * GHZ
        h, _, _, _ = transmon(ej, ec, 0.0, 20)        # 41 charge states: converged
        w = np.linalg.eigvalsh(h)[:4]
        ex = mathieu_transmon_levels(ej, ec, 4)
        assert np.max(np.abs(w - ex)) < 1e-9 * ej


def test_transmon_21_states_converged_against_41():
    ej, ec = 20.0 * GHZ, 0.25 * GHZ
    w21 = np.linalg.eigvalsh(transmon(ej, ec, 0.0, 10)[0])[:4]
    w41 = np.linalg.eigvalsh(transmon(ej, ec, 0.0, 20)[0])[:4]
    assert np.max(np.abs(w21 - w41)) < 1e-7


def test_fluxonium_harmonic_limit():
    # E_J = 0: exact harmonic oscillator, levels omega_p * k
    ec, el = 1.0 * GHZ, 0.9 * GHZ
    m = build_mode({"kind": "fluxonium", "ej": 0.0, "ec": ec, "el": el,
                    "phi_ext": np.pi, "n_osc": 50, "levels": 5})
    wp = np.sqrt(8 * ec * el)
    assert np.max(np.abs(m["E"] - wp * np.arange(5))) < 1e-10 * wp
    # and <k|phi|k+1> = phi_osc sqrt(k+1)/sqrt2 up to the gauge sign
    po = (8 * ec / el) ** 0.25
    off = np.abs(np.diag(m["ops"]["phi"], 1))
    assert np.allclose(off, po * np.sqrt(np.arange(1, 5) / 2.0), atol=1e-12)


def test_fluxonium_paper_frequencies():
    with open(os.path.join(HERE, "golden", "fluxonium_f01.json")) as f:
        gold = json.load(f)
    for md in gold["modes"]:
        m = build_mode({"kind": "fluxonium", "ej": md["ej_GHz"] * GHZ,
                        "ec": md["ec_GHz"] * GHZ, "el": md["el_GHz"] * GHZ,
                        "phi_ext": np.pi, "n_osc": 50, "levels": 4})
        f01 = m["E"][1] / GHZ
        assert abs(f01 - md["f01_GHz"]) < gold["tolerance_GHz"]


def test_fluxonium_basis_converged_50_vs_80():
    spec = {"kind": "fluxonium", "ej": 4.0 * GHZ, "ec": 1.0 * GHZ, "el": 1.0 * GHZ,
            "phi_ext": np.pi, "levels": 5}
    a = build_mode(dict(spec, n_osc=50))
    b = build_mode(dict(spec, n_osc=80))
    assert np.max(np.abs(a["E"] - b["E"])) < 1e-8
    assert np.max(np.abs(np.abs(a["ops"]["phi"]) - np.abs(b["ops"]["phi"]))) < 1e-8


def test_fluxonium_operators_are_hermitian_conjugate_pair():
    m = build_mode({"kind": "fluxonium", "ej": 4 * GHZ, "ec": 1 * GHZ, "el": 1 * GHZ,
                    "phi_ext": np.pi, "n_osc": 50, "levels": 5})
    for X in m["ops"].values():
        assert np.allclose(X, X.conj().T, atol=1e-13)
    # canonical commutator [phi, n] = i holds on the low-lying levels (the
    # truncation only spoils it near the cut-off)
    full = m["full_ops"]
    c = full["phi"] @ full["n"] - full["n"] @ full["phi"]
    assert np.allclose(np.diag(c)[:40], 1j, atol=1e-12)


def test_sweet_spot_operators_are_parity_odd():
    # phi_ext = pi and n_g = 0 make the potential even: n and phi only connect
    # levels of opposite parity
    for spec in [{"kind": "fluxonium", "ej": 4 * GHZ, "ec": 1 * GHZ, "el": 1 * GHZ,
                  "phi_ext": np.pi, "n_osc": 50, "levels": 5},
                 {"kind": "transmon", "ej": 20 * GHZ, "ec": 0.25 * GHZ, "ng": 0.0,
                  "ncut": 10, "levels": 5}]:
        m = build_mode(spec)
        for X in m["ops"].values():
            for a in range(5):
                for b in range(5):
                    if (a + b) % 2 == 0:
                        assert abs(X[a, b]) < 1e-12 * np.max(np.abs(X))


def test_gauge_rule():
    rng = np.random.default_rng(1)
    v = np.linalg.qr(rng.standard_normal((6, 6)))[0]
    g = gauge_fix(v)
    for j in range(6):
        col = g[:, j]
        i = np.nonzero(np.abs(col) >= 1e-3 * np.max(np.abs(col)))[0][0]
        assert col[i] > 0
        assert np.allclose(np.abs(col), np.abs(v[:, j]))


@pytest.mark.parametrize("kind", ["transmon", "fluxonium"])
def test_eigen_derivatives_match_central_differences(kind):
    if kind == "transmon":
        spec = {"kind": kind, "ej": 20 * GHZ, "ec": 0.25 * GHZ, "ng": 0.0, "ncut": 10,
                "levels": 4}
        params = ["ej", "ec"]
    else:
        spec = {"kind": kind, "ej": 4 * GHZ, "ec": 1 * GHZ, "el": 1.1 * GHZ,
                "phi_ext": np.pi, "n_osc": 50, "levels": 4}
        params = ["ej", "ec", "el"]
    m = build_mode(spec)
    for p in params:
        dE, dops = mode_derivatives(m, p)
        h = 1e-6 * spec[p]
        mp = build_mode(dict(spec, **{p: spec[p] + h}))
        mm = build_mode(dict(spec, **{p: spec[p] - h}))
        fdE = (mp["E"] - mm["E"]) / (2 * h)
        assert np.max(np.abs(dE - fdE)) < 1e-6 * max(1.0, np.max(np.abs(fdE)))
        for name in dops:
            fd = (mp["ops"][name] - mm["ops"][name]) / (2 * h)
            assert np.max(np.abs(dops[name] - fd)) < 1e-6 * max(1.0, np.max(np.abs(fd)))
