"""Seeded synthetic inputs for the evolution path.

This module draws parameters and random targets and nothing else: it holds
none of the method's arithmetic (no Hamiltonian, no eigensolve, no evolution,
no fidelity).  Tests feed the same dictionaries to the oracle and to the CUDA
library, and ``bench.py`` times the library on them.

A workload is a plain dict::

    {
      "name": str,
      "modes":     [{"kind": "transmon", "ej", "ec", "ng", "ncut", "levels"} |
                    {"kind": "fluxonium", "ej", "ec", "el", "phi_ext", "n_osc", "levels"}],
                   (optional "coupler": True: held in level 0 in the computational subspace;
                    optional "local_ops": {name: d x d Hermitian matrix in the truncated
                    eigenbasis}, usable as an operator name on that mode)
      "couplings": [{"a", "op_a", "b", "op_b", "J"}],          # op: "n", "phi" or a local name
      "drives":    [{"mode", "op", "env", "amp" | "amps", "sigma", "t0", "length",
                     "omega_d" (float) or "omega_mode" (int), "phase"}],
      "T", "dt", "frame" ("interaction" | "lab"),
      "col_index": [flat product-basis index of each evolved column],
      "target":    complex (Dc, Dc) array, Dc = 2**(number of non-coupler modes),
      "fid_kind":  "avg" | "state",
    }

Units: every energy, amplitude and frequency is angular, in rad/ns.  The paper
quotes them as 2*pi*GHz (Sec. 3.1); GHz inputs are multiplied by 2*pi and MHz
inputs by 2*pi*1e-3.  Times are in ns.

The shapes and value ranges follow the paper's workloads: the two-transmon
gate, the cross-resonance fluxonium pair (Sec. 3.4, App. C), the fluxonium
chain with simultaneous drives (Sec. 4, App. C) and a ring of ten fluxoniums.
"""
import numpy as np

TWO_PI = 2.0 * np.pi
GHZ = TWO_PI
MHZ = TWO_PI * 1e-3


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def haar_unitary(n, rng):
    """Haar-random unitary: QR of a complex Ginibre matrix with the phases of
    R's diagonal moved into Q (Mezzadri's recipe)."""
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def x_all_target(nq):
    """X on every qubit as a (2^nq x 2^nq) permutation matrix (mode 0 = MSB)."""
    dc = 2 ** nq
    t = np.zeros((dc, dc), dtype=np.complex128)
    for j in range(dc):
        t[(dc - 1) ^ j, j] = 1.0
    return t


def comp_flat_index(bits, dims):
    """Flat product-basis index of the bare state with level bits[i] on mode i
    (mode 0 most significant).  Pure index bookkeeping."""
    r = 0
    for b, d in zip(bits, dims):
        r = r * d + int(b)
    return r


def comp_states(dims, couplers=()):
    """Flat indices of the computational states: qubit modes in {0, 1} (first qubit
    most significant), coupler modes (indices in `couplers`) in level 0."""
    qubits = [i for i in range(len(dims)) if i not in set(couplers)]
    out = []
    for j in range(2 ** len(qubits)):
        bits = [0] * len(dims)
        for b, i in enumerate(qubits):
            bits[i] = (j >> (len(qubits) - 1 - b)) & 1
        out.append(comp_flat_index(bits, dims))
    return out


def _fluxonium_mode(rng, levels, n_osc=50):
    return {"kind": "fluxonium", "ej": rng.uniform(3.0, 5.0) * GHZ,
            "ec": rng.uniform(0.8, 1.2) * GHZ, "el": rng.uniform(0.8, 1.2) * GHZ,
            "phi_ext": np.pi, "n_osc": n_osc, "levels": levels}


def _transmon_mode(rng, levels, ncut=10):
    return {"kind": "transmon", "ej": rng.uniform(15.0, 25.0) * GHZ,
            "ec": rng.uniform(0.2, 0.3) * GHZ, "ng": 0.0, "ncut": ncut, "levels": levels}


def _pwc_drive(rng, mode, op, nseg, length, omega_mode):
    return {"mode": mode, "op": op, "env": "pwc",
            "amps": list(rng.uniform(10.0, 50.0, size=nseg) * MHZ),
            "length": length, "omega_mode": omega_mode, "phase": 0.0}


def transmon_pair(seed=0, T=50.0, dt=0.005):
    """Two capacitively coupled transmons, 21 charge states -> 4 levels each
    (D = 16), g on n1 (x) n2, Gaussian-envelope cosine drive on qubit 1 at its
    own 0-1 frequency, all 16 basis states evolved, Haar 4x4 target."""
    rng = _rng(seed)
    modes = [_transmon_mode(rng, 4), _transmon_mode(rng, 4)]
    g = rng.uniform(5.0, 20.0) * MHZ
    amp = rng.uniform(10.0, 50.0) * MHZ
    target = haar_unitary(4, rng)
    return {"name": "transmon_pair_d16", "modes": modes,
            "couplings": [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": g}],
            "drives": [{"mode": 0, "op": "n", "env": "gaussian", "amp": amp,
                        "sigma": T / 4.0, "t0": T / 2.0, "length": T,
                        "omega_mode": 0, "phase": 0.0}],
            "T": T, "dt": dt, "frame": "interaction",
            "col_index": list(range(16)), "target": target, "fid_kind": "avg"}


def fluxonium_pair_cr(seed=0, T=100.0, dt=0.01, nseg=20):
    """Two fluxoniums (50 oscillator states -> 5 levels, D = 25), J on n1 (x) n2,
    cross-resonance style flux drive on qubit 1 at qubit 2's 0-1 frequency,
    piecewise-constant envelope; the 4 computational states are evolved."""
    rng = _rng(seed)
    modes = [_fluxonium_mode(rng, 5), _fluxonium_mode(rng, 5)]
    J = rng.uniform(10.0, 30.0) * MHZ
    drive = _pwc_drive(rng, 0, "phi", nseg, T, omega_mode=1)
    target = haar_unitary(4, rng)
    dims = [5, 5]
    return {"name": "fluxonium_pair_cr_d25", "modes": modes,
            "couplings": [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": J}],
            "drives": [drive], "T": T, "dt": dt, "frame": "interaction",
            "col_index": comp_states(dims), "target": target, "fid_kind": "avg"}


def fluxonium_pair_multipath(seed=0, T=50.0, dt=0.01, nseg=10, levels=4):
    """Two fluxoniums with the multipath coupling of Sec. 3.1, J_C n1 n2 - J_L phi1 phi2
    (J_C ~ U[10, 30] MHz, J_L ~ U[0.5, 2] MHz: a capacitive and an inductive term on
    the same pair), PWC flux drives on both qubits at their own 0-1 frequencies,
    Haar target, all computational states."""
    rng = _rng(seed)
    modes = [_fluxonium_mode(rng, levels), _fluxonium_mode(rng, levels)]
    jc = rng.uniform(10.0, 30.0) * MHZ
    jl = rng.uniform(0.5, 2.0) * MHZ
    drives = [_pwc_drive(rng, i, "phi", nseg, T, omega_mode=i) for i in range(2)]
    dims = [levels, levels]
    return {"name": f"fluxonium_multipath_l{levels}", "modes": modes,
            "couplings": [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": jc},
                          {"a": 0, "op_a": "phi", "b": 1, "op_b": "phi", "J": -jl}],
            "drives": drives, "T": T, "dt": dt, "frame": "interaction",
            "col_index": comp_states(dims), "target": haar_unitary(4, rng), "fid_kind": "avg"}


def local_op_pair(seed=0, T=30.0, dt=0.01, nseg=10, levels=4):
    """Two fluxoniums with generic Kronecker terms (Eq. 1) built from local operators
    given in the truncated eigenbasis: a drive on qubit 0 through sx = |0><1| + |1><0|
    (parity-odd), a seeded random Hermitian h on each mode (no parity structure,
    entries ~ 0.1) coupled as J_h h (x) h with J_h ~ U[1, 5] MHz next to the n (x) n
    coupling, and a PWC flux drive on qubit 1; Haar target."""
    rng = _rng(seed)
    modes = [_fluxonium_mode(rng, levels), _fluxonium_mode(rng, levels)]
    sx = np.zeros((levels, levels), dtype=np.complex128)
    sx[0, 1] = sx[1, 0] = 1.0
    for m in modes:
        g = (rng.standard_normal((levels, levels)) + 1j * rng.standard_normal((levels, levels))) * 0.05
        m["local_ops"] = {"sx": sx.copy(), "h": g + g.conj().T}
    couplings = [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": rng.uniform(10.0, 30.0) * MHZ},
                 {"a": 0, "op_a": "h", "b": 1, "op_b": "h", "J": rng.uniform(1.0, 5.0) * MHZ}]
    drives = [_pwc_drive(rng, 0, "sx", nseg, T, omega_mode=0),
              _pwc_drive(rng, 1, "phi", nseg, T, omega_mode=1)]
    dims = [levels, levels]
    return {"name": f"local_op_pair_l{levels}", "modes": modes, "couplings": couplings,
            "drives": drives, "T": T, "dt": dt, "frame": "interaction",
            "col_index": comp_states(dims), "target": haar_unitary(4, rng), "fid_kind": "avg"}


def coupler_scheme(seed=0, kind="ftf", T=40.0, dt=0.01, nseg=10, levels=(4, 4, 4)):
    """Two qubits interacting through a transmon coupler in the middle (Sec. 4: "ttt",
    transmon qubits with a transmon coupler; "ftf", fluxonium qubits with a transmon
    coupler).  Qubit-coupler couplings n (x) n with g ~ U[20, 60] MHz and a weaker
    direct qubit-qubit n (x) n term (U[1, 5] MHz); PWC drives on the two qubits at
    their own 0-1 frequencies; the coupler is undriven and held in its ground state
    in the computational subspace (4 states); Haar 4 x 4 target."""
    rng = _rng(seed)
    qubit = _fluxonium_mode if kind == "ftf" else _transmon_mode
    op = "phi" if kind == "ftf" else "n"
    modes = [qubit(rng, levels[0]), dict(_transmon_mode(rng, levels[1]), coupler=True),
             qubit(rng, levels[2])]
    couplings = [{"a": 0, "op_a": "n", "b": 1, "op_b": "n", "J": rng.uniform(20.0, 60.0) * MHZ},
                 {"a": 1, "op_a": "n", "b": 2, "op_b": "n", "J": rng.uniform(20.0, 60.0) * MHZ},
                 {"a": 0, "op_a": "n", "b": 2, "op_b": "n", "J": rng.uniform(1.0, 5.0) * MHZ}]
    drives = [_pwc_drive(rng, i, op, nseg, T, omega_mode=i) for i in (0, 2)]
    dims = list(levels)
    return {"name": f"{kind}_l{'_'.join(map(str, levels))}", "modes": modes,
            "couplings": couplings, "drives": drives, "T": T, "dt": dt, "frame": "interaction",
            "col_index": comp_states(dims, couplers=(1,)), "target": haar_unitary(4, rng),
            "fid_kind": "avg"}


def fluxonium_chain(seed=0, nq=6, levels=4, T=60.0, dt=0.01, nseg=10, ring=False,
                    ncols=None):
    """Chain (or ring) of fluxoniums with nearest-neighbour n (x) n couplings and a
    piecewise-constant flux drive on every qubit at its own 0-1 frequency;
    target X on every qubit.  ncols=None evolves every computational state,
    otherwise ncols distinct seeded computational bitstrings."""
    rng = _rng(seed)
    modes = [_fluxonium_mode(rng, levels) for _ in range(nq)]
    edges = [(i, i + 1) for i in range(nq - 1)] + ([(nq - 1, 0)] if ring else [])
    couplings = [{"a": a, "op_a": "n", "b": b, "op_b": "n",
                  "J": rng.uniform(10.0, 30.0) * MHZ} for a, b in edges]
    drives = [_pwc_drive(rng, i, "phi", nseg, T, omega_mode=i) for i in range(nq)]
    dims = [levels] * nq
    comp = comp_states(dims)
    if ncols is None:
        cols = comp
    else:
        pick = rng.choice(len(comp), size=ncols, replace=False)
        cols = [comp[int(j)] for j in sorted(pick)]
    return {"name": f"fluxonium_{'ring' if ring else 'chain'}{nq}_l{levels}",
            "modes": modes, "couplings": couplings, "drives": drives,
            "T": T, "dt": dt, "frame": "interaction", "col_index": cols,
            "target": x_all_target(nq), "fid_kind": "state"}


def fluxonium_chain6(seed=0, T=60.0, dt=0.01):
    """6-fluxonium chain, 4 levels (D = 4096), all 64 computational states."""
    return fluxonium_chain(seed=seed, nq=6, levels=4, T=T, dt=dt, nseg=10)


def fluxonium_ring10(seed=0, T=40.0, dt=0.01, ncols=16):
    """10-fluxonium ring, 4 levels (D = 1,048,576), 16 seeded computational states."""
    return fluxonium_chain(seed=seed, nq=10, levels=4, T=T, dt=dt, nseg=10,
                           ring=True, ncols=ncols)


def serving_request(rng, dt=0.01, nq=None, kind=None, levels=None):
    """One request of the serving stream: 2-5 coupled transmons or fluxoniums
    (one kind per request), 3-5 levels, T ~ U[20, 200] ns rounded to whole
    steps, 10-segment random drives on every qubit, all computational states,
    Haar target, fidelity plus gradient.  nq, kind and levels fix the request's
    shape (the same random draws are made either way)."""
    nq_draw = int(rng.integers(2, 6))
    kind_draw = "transmon" if rng.integers(0, 2) == 0 else "fluxonium"
    levels_draw = int(rng.integers(3, 6))
    nq = nq_draw if nq is None else nq
    kind = kind_draw if kind is None else kind
    levels = levels_draw if levels is None else levels
    nsteps = int(round(rng.uniform(20.0, 200.0) / dt))
    T = nsteps * dt
    if kind == "transmon":
        modes = [_transmon_mode(rng, levels) for _ in range(nq)]
        op = "n"
    else:
        modes = [_fluxonium_mode(rng, levels) for _ in range(nq)]
        op = "phi"
    couplings = [{"a": i, "op_a": "n", "b": i + 1, "op_b": "n",
                  "J": rng.uniform(5.0, 30.0) * MHZ} for i in range(nq - 1)]
    drives = [_pwc_drive(rng, i, op, 10, T, omega_mode=i) for i in range(nq)]
    dims = [levels] * nq
    return {"name": f"req_{kind}{nq}_l{levels}", "modes": modes,
            "couplings": couplings, "drives": drives, "T": T, "dt": dt,
            "frame": "interaction", "col_index": comp_states(dims),
            "target": haar_unitary(2 ** nq, rng), "fid_kind": "avg"}


def serving_stream(seed=0, n=10000, rate=1.0):
    """Poisson arrivals (exponential gaps of mean 1/rate seconds) of serving requests."""
    rng = _rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += rng.exponential(1.0 / rate)
        out.append((t, serving_request(rng)))
    return out


def random_columns(D, S, seed=0):
    """Seeded random normalised complex columns (D x S), for tests that start from
    arbitrary states instead of basis states."""
    rng = _rng(seed)
    z = rng.standard_normal((D, S)) + 1j * rng.standard_normal((D, S))
    return z / np.linalg.norm(z, axis=0, keepdims=True)


CONFIGS = {
    "transmon_pair": transmon_pair,
    "fluxonium_pair_cr": fluxonium_pair_cr,
    "fluxonium_chain6": fluxonium_chain6,
    "fluxonium_ring10": fluxonium_ring10,
}
