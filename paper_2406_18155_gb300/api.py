"""Thin Python layer over the C ABI (argument marshalling only).

PyTorch provides device memory and the stream; every computation runs in the
library's CUDA kernels.
"""
import ctypes as C

import numpy as np

from . import capi
from .capi import check, lib

_OPS = {"n": capi.SG_OP_N, "phi": capi.SG_OP_PHI}
_ENV = {"gaussian": capi.SG_ENV_GAUSSIAN, "pwc": capi.SG_ENV_PWC, "cosine": capi.SG_ENV_COSINE}
_PREC = {"fp64": capi.SG_FP64, "mixed": capi.SG_MIXED}
_FRAME = {"interaction": capi.SG_FRAME_INTERACTION, "lab": capi.SG_FRAME_LAB}
_KIND = {"avg": capi.SG_FID_AVG, "state": capi.SG_FID_STATE}


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c128_pairs(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).view(np.float64)


class Context:
    """sg_ctx on one CUDA device, ordered on a torch stream (current stream by default)."""

    def __init__(self, device=0, stream=None):
        import torch
        self.device = device
        if stream is None:
            with torch.cuda.device(device):
                stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        check(lib().sg_ctx_create(C.byref(h), device, C.c_void_p(stream.cuda_stream)))
        self.h = h

    def close(self):
        if self.h:
            lib().sg_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_SOLVER = {"rk4": capi.SG_SOLVER_RK4, "q1": capi.SG_SOLVER_Q1, "q2": capi.SG_SOLVER_Q2, "q4": capi.SG_SOLVER_Q4,
           "q4j": capi.SG_SOLVER_Q4J}
_COMP = {"none": capi.SG_COMP_NONE, "vz": capi.SG_COMP_VZ}
_BASIS = {"product": capi.SG_BASIS_PRODUCT, "dressed": capi.SG_BASIS_DRESSED}


def evolve_opts(T, dt, precision="mixed", frame="interaction", col_index=None, ncols=None, solver="rk4",
                compensation="none", basis="product"):
    o = capi.sg_evolve_opts()
    o.T, o.dt = float(T), float(dt)
    o.precision = _PREC[precision]
    o.frame = _FRAME[frame]
    o.solver = _SOLVER[solver]
    o.compensation = _COMP[compensation]
    o.basis = _BASIS[basis]
    keep = None
    if col_index is not None:
        keep = np.ascontiguousarray(np.asarray(col_index, dtype=np.int64))
        o.ncols = keep.size
        o.col_index = keep.ctypes.data_as(C.POINTER(C.c_longlong))
    else:
        o.ncols = int(ncols or 0)
        o.col_index = None
    return o, keep


class System:
    def __init__(self, ctx):
        self.ctx = ctx
        h = C.c_void_p()
        check(lib().sg_system_create(ctx.h, C.byref(h)), ctx.h)
        self.h = h
        self._keep = []
        self._local = {}              # (mode, name) -> operator id of a local operator

    def _chk(self, rc):
        return check(rc, self.ctx.h)

    def _op(self, mode, op):
        """Operator id: "n", "phi", a local operator's name on this mode, or an id."""
        if isinstance(op, (int, np.integer)):
            return int(op)
        if op in _OPS:
            return _OPS[op]
        return self._local[(mode, op)]

    def add_local_op(self, mode, matrix, name=None):
        """A d x d Hermitian operator of `mode` in its truncated eigenbasis
        (sg_add_local_op); returns its id, usable by add_drive / add_coupling
        (by id, or by `name`)."""
        a = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128))
        buf = np.ascontiguousarray(a.view(np.float64).reshape(-1))
        k = C.c_int()
        self._chk(lib().sg_add_local_op(self.h, mode, buf.ctypes.data_as(C.POINTER(C.c_double)), C.byref(k)))
        if name is not None:
            self._local[(mode, name)] = k.value
        return k.value

    # --- definition -----------------------------------------------------------
    def add_transmon(self, ej, ec, ng=0.0, ncut=10, levels=4):
        m = C.c_int()
        self._chk(lib().sg_add_transmon(self.h, ej, ec, ng, ncut, levels, C.byref(m)))
        return m.value

    def add_fluxonium(self, ej, ec, el, phi_ext=np.pi, n_osc=50, levels=4):
        m = C.c_int()
        self._chk(lib().sg_add_fluxonium(self.h, ej, ec, el, phi_ext, n_osc, levels, C.byref(m)))
        return m.value

    def add_coupling(self, a, op_a, b, op_b, J):
        t = C.c_int()
        self._chk(lib().sg_add_coupling(self.h, a, self._op(a, op_a), b, self._op(b, op_b), J, C.byref(t)))
        return t.value

    def set_coupler(self, mode, coupler=True):
        """Hold `mode` in its ground state in the computational subspace (sg_set_coupler)."""
        self._chk(lib().sg_set_coupler(self.h, mode, 1 if coupler else 0))

    def add_drive(self, mode, op, env, amp=0.0, amps=None, sigma=1.0, t0=0.0, length=1.0,
                  omega_d=0.0, omega_mode=None, phase=0.0):
        p = capi.sg_pulse()
        p.kind = _ENV[env]
        if amps is not None:
            arr = np.ascontiguousarray(np.asarray(amps, dtype=np.float64))
            self._keep.append(arr)
            p.nseg = arr.size
            p.amps = _dptr(arr)
        else:
            p.nseg = 1
        p.amp, p.sigma, p.t0, p.length = float(amp), float(sigma), float(t0), float(length)
        p.omega_d = float(omega_d) if omega_d is not None else 0.0
        p.omega_mode = -1 if omega_mode is None else int(omega_mode)
        p.phase = float(phase)
        k = C.c_int()
        self._chk(lib().sg_add_drive(self.h, mode, self._op(mode, op), C.byref(p), C.byref(k)))
        return k.value

    @classmethod
    def from_workload(cls, ctx, wl):
        s = cls(ctx)
        for m in wl["modes"]:
            if m["kind"] == "transmon":
                s.add_transmon(m["ej"], m["ec"], m.get("ng", 0.0), m.get("ncut", 10), m["levels"])
            else:
                s.add_fluxonium(m["ej"], m["ec"], m["el"], m.get("phi_ext", np.pi),
                                m.get("n_osc", 50), m["levels"])
        for i, m in enumerate(wl["modes"]):
            if m.get("coupler"):
                s.set_coupler(i, True)
            for name, mat in m.get("local_ops", {}).items():
                s.add_local_op(i, mat, name)
        for c in wl["couplings"]:
            s.add_coupling(c["a"], c["op_a"], c["b"], c["op_b"], c["J"])
        for d in wl["drives"]:
            s.add_drive(d["mode"], d["op"], d["env"], amp=d.get("amp", 0.0), amps=d.get("amps"),
                        sigma=d.get("sigma", 1.0), t0=d.get("t0", 0.0), length=d["length"],
                        omega_d=d.get("omega_d", 0.0), omega_mode=d.get("omega_mode"),
                        phase=d.get("phase", 0.0))
        for c in wl.get("collapse", []):
            s.add_collapse(c["mode"], c["L"], c["rate"])
        s.wl = wl
        return s

    def add_collapse(self, mode, L, rate):
        """Collapse operator L (d x d, truncated eigenbasis) on `mode` at rate (1/ns)."""
        a = _c128_pairs(np.asarray(L, dtype=np.complex128))
        self._keep.append(a)
        out = C.c_int()
        self._chk(lib().sg_add_collapse(self.h, int(mode), _dptr(a), float(rate), C.byref(out)))
        return out.value

    def evolve_open(self, T, dt, rho0, precision="mixed", frame="interaction"):
        """Lab-frame rho(T) (D x D numpy) of the open evolution from rho0 (sg_evolve_open)."""
        o, keep = evolve_opts(T, dt, precision, frame, None, ncols=1)
        r0 = _c128_pairs(np.asarray(rho0, dtype=np.complex128))
        out = np.zeros_like(r0)
        self._chk(lib().sg_evolve_open(self.h, C.byref(o), _dptr(r0), _dptr(out)))
        return out.view(np.complex128).reshape(np.asarray(rho0).shape)

    def gate_fidelity_open(self, T, dt, target, precision="mixed", frame="interaction"):
        """(F_avg, F_pro) of the open evolution on the computational block against the
        target unitary (sg_gate_fidelity_open)."""
        o, keep = evolve_opts(T, dt, precision, frame, None, ncols=1)
        tg = _c128_pairs(target)
        F = np.zeros(2)
        self._chk(lib().sg_gate_fidelity_open(self.h, C.byref(o), _dptr(tg), _dptr(F)))
        return F[0], F[1]

    def gate_fidelity_open_grad(self, T, dt, target, kind="avg", precision="mixed", frame="interaction", ckpt=0,
                                ham=False):
        """(F_avg, F_pro), dF/d(pulse parameters) and (ham=True) dF/d(Hamiltonian
        parameters, else None) of F_avg (kind "avg") or F_pro (kind "pro") of the open
        evolution (sg_gate_fidelity_open_grad)."""
        o, keep = evolve_opts(T, dt, precision, frame, None, ncols=1)
        tg = _c128_pairs(target)
        F = np.zeros(2)
        npul, nham = self.param_counts()
        g = np.zeros(max(npul, 1))
        gh = np.zeros(max(nham, 1))
        k = {"avg": 0, "pro": 1}[kind]
        self._chk(lib().sg_gate_fidelity_open_grad(self.h, C.byref(o), _dptr(tg), k, _dptr(F), _dptr(g),
                                                   _dptr(gh) if ham else None, int(ckpt)))
        return (F, g[:npul], gh[:nham]) if ham else (F, g[:npul])

    def close(self):
        if self.h:
            lib().sg_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- prepare / inspect --------------------------------------------------------
    def prepare(self):
        self._chk(lib().sg_prepare(self.h))

    def dims(self):
        D, n = C.c_longlong(), C.c_int()
        self._chk(lib().sg_dims(self.h, C.byref(D), C.byref(n)))
        return D.value, n.value

    def spectrum(self, mode, d):
        E = np.zeros(d)
        n = np.zeros(2 * d * d)
        phi = np.zeros(2 * d * d)
        self._chk(lib().sg_get_spectrum(self.h, mode, _dptr(E), _dptr(n), _dptr(phi)))
        return E, n.view(np.complex128).reshape(d, d), phi.view(np.complex128).reshape(d, d)

    def param_counts(self):
        a, b = C.c_int(), C.c_int()
        self._chk(lib().sg_param_counts(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def get_params(self):
        npul, nham = self.param_counts()
        p, h = np.zeros(max(npul, 1)), np.zeros(max(nham, 1))
        self._chk(lib().sg_get_params(self.h, _dptr(p), _dptr(h)))
        return p[:npul], h[:nham]

    def set_params(self, pulse=None, ham=None):
        pa = None if pulse is None else np.ascontiguousarray(np.asarray(pulse, dtype=np.float64))
        ha = None if ham is None else np.ascontiguousarray(np.asarray(ham, dtype=np.float64))
        self._chk(lib().sg_set_params(self.h, None if pa is None else _dptr(pa),
                                      None if ha is None else _dptr(ha)))

    # --- evolution -----------------------------------------------------------------
    def evolve(self, T, dt, precision="mixed", frame="interaction", col_index=None, psi=None, solver="rk4"):
        """Lab-frame columns after T, as a (D, S) complex128 torch tensor on the device.
        Starts from basis states col_index, or from the given device tensor psi.
        solver: "rk4", or the Suzuki-Trotter "q1", "q2", "q4", "q4j" (App. A; lab frame)."""
        import torch
        D, _ = self.dims()
        if psi is None:
            S = len(col_index)
            psi = torch.empty((D, S), dtype=torch.complex128, device=f"cuda:{self.ctx.device}")
            o, keep = evolve_opts(T, dt, precision, frame, col_index, solver=solver)
        else:
            assert psi.dtype == torch.complex128 and psi.is_contiguous() and psi.shape[0] == D
            o, keep = evolve_opts(T, dt, precision, frame, None, ncols=psi.shape[1], solver=solver)
        self._chk(lib().sg_evolve(self.h, C.byref(o), C.c_void_p(psi.data_ptr())))
        return psi

    def fidelity(self, T, dt, target, col_index, precision="mixed", frame="interaction", solver="rk4",
                 compensation="none", basis="product"):
        """(F_avg, F_state, computational block); compensation "vz": the fidelities with
        the virtual Z gates around the pulses that maximise them; basis "dressed": the
        gate in the eigenbasis of the idle Hamiltonian."""
        o, keep = evolve_opts(T, dt, precision, frame, col_index, solver=solver, compensation=compensation,
                              basis=basis)
        tg = _c128_pairs(target)
        F = np.zeros(2)
        Dc = target.shape[0]
        U = np.zeros(2 * Dc * len(col_index))
        self._chk(lib().sg_fidelity(self.h, C.byref(o), _dptr(tg), _dptr(F), _dptr(U)))
        return F[0], F[1], U.view(np.complex128).reshape(Dc, len(col_index))

    def fidelity_grad(self, T, dt, target, col_index, kind="avg", precision="mixed",
                      frame="interaction", ckpt=0, ham=True, solver="rk4", compensation="none",
                      basis="product"):
        """F and the gradient w.r.t. the pulse and (ham=True) Hamiltonian parameters;
        with ham=False the Hamiltonian part is not computed and returned as None.
        solver "q2", "q4" or "q4j" (lab frame) computes the pulse-parameter gradient only: pass ham=False.
        compensation "vz": F with the virtual Z gates that maximise it, and its gradient;
        basis "dressed" (pulse gradient only: ham=False): the gate in the idle eigenbasis."""
        o, keep = evolve_opts(T, dt, precision, frame, col_index, solver=solver, compensation=compensation,
                              basis=basis)
        tg = _c128_pairs(target)
        F = np.zeros(2)
        npul, nham = self.param_counts()
        gp, gh = np.zeros(max(npul, 1)), np.zeros(max(nham, 1))
        self._chk(lib().sg_fidelity_grad(self.h, C.byref(o), _dptr(tg), _KIND[kind], _dptr(F),
                                         _dptr(gp), _dptr(gh) if ham else None, int(ckpt)))
        return F, gp[:npul], (gh[:nham] if ham else None)

    def fidelity_grad_sharded(self, T, dt, target, col_index, allreduce, kind="avg", precision="mixed",
                              frame="interaction", ckpt=0, ham=True, solver="rk4"):
        """This shard's part of a column-sharded fidelity + gradient solve
        (sg_fidelity_grad_sharded): col_index are this shard's columns, `allreduce` maps
        a float64 numpy vector to its sum over all shards (shard.torch_allreduce).
        Returns the F and gradient of the whole solve, the same on every shard."""
        from .capi import SG_ALLREDUCE_FN
        o, keep = evolve_opts(T, dt, precision, frame, col_index, solver=solver)
        tg = _c128_pairs(target)
        F = np.zeros(2)
        npul, nham = self.param_counts()
        gp, gh = np.zeros(max(npul, 1)), np.zeros(max(nham, 1))

        def cb(buf, n, user):
            try:
                v = np.ctypeslib.as_array(buf, shape=(n,))
                v[:] = np.asarray(allreduce(v.copy()), dtype=np.float64).reshape(n)
                return 0
            except Exception:                      # reported by the library as SG_E_STATE
                return 1
        fn = SG_ALLREDUCE_FN(cb)
        self._chk(lib().sg_fidelity_grad_sharded(self.h, C.byref(o), _dptr(tg), _KIND[kind], _dptr(F),
                                                 _dptr(gp), _dptr(gh) if ham else None, int(ckpt), fn, None))
        return F, gp[:npul], (gh[:nham] if ham else None)

    def last_stats(self):
        out = np.zeros(5)
        self._chk(lib().sg_last_stats(self.h, _dptr(out)))
        return {"forward_ms": out[0], "backward_ms": out[1], "peak_bytes": out[2],
                "ckpt_interval": int(out[3]), "launches": int(out[4])}


def evolve_batch(systems, T, dt, col_index, frame="interaction"):
    """Lab-frame states of prepared same-shape systems evolved together on the tensor
    cores (sg_evolve_batch): a (B, D, S) complex128 torch tensor on the device."""
    import torch
    D, _ = systems[0].dims()
    S = len(col_index)
    psi = torch.empty((len(systems), D, S), dtype=torch.complex128, device=f"cuda:{systems[0].ctx.device}")
    o, keep = evolve_opts(T, dt, "mixed", frame, col_index)
    hs = (C.c_void_p * len(systems))(*[s.h for s in systems])
    systems[0]._chk(lib().sg_evolve_batch(hs, len(systems), C.byref(o), C.c_void_p(psi.data_ptr())))
    return psi


def workload_fidelity(ctx, wl, precision="mixed", grad=False, ckpt=0):
    """Convenience: build, prepare and solve one workload dict."""
    s = System.from_workload(ctx, wl)
    s.prepare()
    if grad:
        F, gp, gh = s.fidelity_grad(wl["T"], wl["dt"], wl["target"], wl["col_index"],
                                    kind=wl["fid_kind"], precision=precision,
                                    frame=wl.get("frame", "interaction"), ckpt=ckpt)
        return s, F, gp, gh
    Fa, Fs, U = s.fidelity(wl["T"], wl["dt"], wl["target"], wl["col_index"], precision=precision,
                           frame=wl.get("frame", "interaction"))
    return s, (Fa, Fs), U


class Server:
    """Continuous-batching server (sg_server_*): requests are admitted by device
    memory and free slots, and run concurrently on the slots' streams; with
    max_batch > 1 a slot packs queued same-shape requests into shared batched
    launches (sg_server_set_batch)."""

    def __init__(self, ctx, mem_budget_bytes, max_slots, max_batch=1):
        self.ctx = ctx
        h = C.c_void_p()
        check(lib().sg_server_create(ctx.h, C.c_size_t(int(mem_budget_bytes)), int(max_slots),
                                     C.byref(h)), ctx.h)
        self.h = h
        self._keep = {}
        if max_batch > 1:
            check(lib().sg_server_set_batch(self.h, int(max_batch)), ctx.h)

    def submit(self, system, T, dt, target, col_index=None, kind="avg", precision="mixed",
               want_grad=True):
        r = capi.sg_request()
        r.sys = system.h
        o, keep = evolve_opts(T, dt, precision, "interaction", col_index, ncols=0)
        r.opts = o
        tg = _c128_pairs(target)
        r.target_re_im = _dptr(tg)
        r.kind = _KIND[kind]
        r.want_grad = 1 if want_grad else 0
        t = C.c_uint64()
        check(lib().sg_server_submit(self.h, C.byref(r), C.byref(t)), self.ctx.h)
        self._keep[t.value] = (system, keep, tg)
        return t.value

    def _result(self, res):
        out = {"status": res.status, "F": (res.F[0], res.F[1]), "submit_s": res.submit_s,
               "start_s": res.start_s, "done_s": res.done_s,
               "error": res.error.decode(errors="replace")}
        out["grad_pulse"] = np.array([res.grad_pulse[i] for i in range(res.n_pulse)])
        out["grad_ham"] = np.array([res.grad_ham[i] for i in range(res.n_ham)])
        return out

    def poll(self, ticket):
        res = capi.sg_result()
        rc = lib().sg_server_poll(self.h, C.c_uint64(ticket), C.byref(res))
        if rc == capi.SG_E_PENDING:
            return None
        check(rc, self.ctx.h)
        return self._result(res)

    def wait(self, ticket):
        res = capi.sg_result()
        check(lib().sg_server_wait(self.h, C.c_uint64(ticket), C.byref(res)), self.ctx.h)
        return self._result(res)

    def cancel(self, ticket):
        return lib().sg_server_cancel(self.h, C.c_uint64(ticket))

    def stats(self):
        st = capi.sg_stats()
        check(lib().sg_server_stats(self.h, C.byref(st)), self.ctx.h)
        return {f: getattr(st, f) for f, _ in capi.sg_stats._fields_}

    def close(self):
        if self.h:
            lib().sg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
