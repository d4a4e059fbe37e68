"""Python binding of libqed (include/qed.h): argument marshalling only.

Every step of the master-equation path runs in the library's CUDA kernels; PyTorch
supplies device memory and streams.  There is no CPU fallback: if libqed.so is missing
or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqed.so")

QED_OK, QED_EINVAL, QED_ENOMEM, QED_ECUDA, QED_ETIMEOUT, QED_ENUMERIC, QED_EUNSUPPORTED = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ETIMEOUT", "ENUMERIC", "EUNSUPPORTED"]
PRECISIONS = {"fp64": 0, "split_fp16x2": 1, "split_bf16x3": 2, "split_tf32x3": 3}
SCHEMES = {"lie": 0, "strang": 1, "effective": 2}

_c_int32_p = ctypes.POINTER(ctypes.c_int32)
_c_double_p = ctypes.POINTER(ctypes.c_double)


class QedError(RuntimeError):
    def __init__(self, status, where, message):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 7 else status}: {message}")


class QedSpec(ctypes.Structure):
    _fields_ = [
        ("n_cavities", ctypes.c_int32),
        ("atoms_per_cavity", _c_int32_p),
        ("n_max", _c_int32_p),
        ("n_extra", ctypes.c_int32),
        ("basis_kind", ctypes.c_int32),
        ("excitation_cap", ctypes.c_int32),
        ("dim_cap", ctypes.c_int64),
        ("omega_c", ctypes.c_double),
        ("omega_a", ctypes.c_double),
        ("g", _c_double_p),
        ("n_bonds", ctypes.c_int32),
        ("bond_ij", _c_int32_p),
        ("zeta", _c_double_p),
        ("extra_tunnel", _c_double_p),
        ("n_jumps", ctypes.c_int32),
        ("jump_kind", _c_int32_p),
        ("jump_site", _c_int32_p),
        ("gamma", _c_double_p),
    ]


_lib = None


def lib():
    """The loaded libqed.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libqed.so is not built; run paper_2403_07042_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "qed_spec_dim": [ctypes.POINTER(QedSpec), ctypes.POINTER(i64), _c_int32_p],
        "qed_spec_basis": [ctypes.POINTER(QedSpec), _c_int32_p, i64],
        "qed_spec_hamiltonian": [ctypes.POINTER(QedSpec), _c_double_p, i64],
        "qed_spec_jump": [ctypes.POINTER(QedSpec), i32, _c_double_p, i64],
        "qed_spec_restricted": [ctypes.POINTER(QedSpec), ctypes.POINTER(i64), i64, i32, _c_double_p, i64,
                                _c_double_p],
        "qed_build": [ctypes.POINTER(QedSpec), dbl, i32, vp, ctypes.POINTER(vp)],
        "qed_free": [vp],
        "qed_dim": [vp, ctypes.POINTER(i64)],
        "qed_basis_labels": [vp, _c_int32_p],
        "qed_basis_index": [vp, _c_int32_p, ctypes.POINTER(i64)],
        "qed_n_observables": [vp, _c_int32_p],
        "qed_set_renorm_every": [vp, i32],
        "qed_set_scheme": [vp, i32],
        "qed_autotune": [vp, i32, ctypes.c_char_p, i32, vp],
        "qed_autotune_batched": [i32, ctypes.POINTER(vp), i32, ctypes.c_char_p, i32, vp],
        "qed_set_plan": [vp, i32, i32, i32, i32, vp],
        "qed_evolve": [vp, vp, i64, i64, i32, i32, _c_int32_p, vp, vp],
        "qed_observables": [vp, vp, i32, _c_int32_p, vp, vp],
        "qed_sync_status": [vp, vp],
        "qed_set_U": [vp, vp, vp],
        "qed_get_U": [vp, vp, vp],
        "qed_profile": [vp, vp, i64, _c_double_p, i32, ctypes.c_char_p, i32, vp],
        "qed_launch_count": [ctypes.POINTER(i64)],
        "qed_profile_replay": [vp, vp, i32, _c_double_p, i32, ctypes.c_char_p, i32, vp],
        "qed_adjoint": [vp, vp, i64, i32, vp, vp, vp, vp, vp, vp],
        "qed_evolve_batched": [i32, ctypes.POINTER(vp), ctypes.POINTER(vp), i64, i32, ctypes.POINTER(vp), vp],
        "qed_select_states": [vp, vp, i64, i32, dbl, ctypes.POINTER(vp), vp, ctypes.POINTER(i64),
                              ctypes.POINTER(i64), ctypes.POINTER(i64), vp],
        "qed_tc_gemm": [vp, i32, vp, i32, i32, i32, i32, i32, _c_int32_p, i32, vp, vp],
        "qed_tc_gemm_static": [vp, i32, vp, i32, i32, i32, i32, i32, _c_int32_p, i32, vp, vp],
        "qed_set_wait_gate": [vp, i32, i64, vp],
        "qed_set_alloc_budget": [i64],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.qed_last_error.argtypes = []
    L.qed_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status, where):
    if status != QED_OK:
        raise QedError(status, where, lib().qed_last_error().decode(errors="replace"))


def _arr(values, ctype):
    a = np.ascontiguousarray(np.asarray(values, dtype=ctype))
    if a.size == 0:
        a = np.zeros(1, dtype=ctype)
    return a


def make_spec(model):
    """A qed_spec for a model dictionary (see qed_workloads); returns (spec, keepalive)."""
    keep = {
        "apc": _arr(model["atoms_per_cavity"], np.int32),
        "nmax": _arr(model["n_max"], np.int32),
        "g": _arr(model["g"], np.float64),
        "bonds": _arr([x for b in model["bonds"] for x in b], np.int32),
        "zeta": _arr(model["zeta"], np.float64),
        "tun": _arr(model["extra_tunnel"], np.float64),
        "jk": _arr([j[0] for j in model["jumps"]], np.int32),
        "js": _arr([j[1] for j in model["jumps"]], np.int32),
        "jg": _arr([j[2] for j in model["jumps"]], np.float64),
    }
    p = lambda a, t: a.ctypes.data_as(t)
    s = QedSpec(
        n_cavities=model["n_cavities"], atoms_per_cavity=p(keep["apc"], _c_int32_p),
        n_max=p(keep["nmax"], _c_int32_p), n_extra=model["n_extra"], basis_kind=model["basis_kind"],
        excitation_cap=model["excitation_cap"], dim_cap=model["dim_cap"],
        omega_c=model["omega_c"], omega_a=model["omega_a"], g=p(keep["g"], _c_double_p),
        n_bonds=len(model["bonds"]), bond_ij=p(keep["bonds"], _c_int32_p),
        zeta=p(keep["zeta"], _c_double_p), extra_tunnel=p(keep["tun"], _c_double_p),
        n_jumps=len(model["jumps"]), jump_kind=p(keep["jk"], _c_int32_p),
        jump_site=p(keep["js"], _c_int32_p), gamma=p(keep["jg"], _c_double_p),
    )
    return s, keep


def spec_dim(model):
    s, _k = make_spec(model)
    d, nd = ctypes.c_int64(), ctypes.c_int32()
    _check(lib().qed_spec_dim(ctypes.byref(s), ctypes.byref(d), ctypes.byref(nd)), "qed_spec_dim")
    return d.value, nd.value


def spec_basis(model):
    D, nd = spec_dim(model)
    s, _k = make_spec(model)
    out = np.zeros((D, nd), dtype=np.int32)
    _check(lib().qed_spec_basis(ctypes.byref(s), out.ctypes.data_as(_c_int32_p), out.size), "qed_spec_basis")
    return out


def spec_hamiltonian(model):
    D, _ = spec_dim(model)
    s, _k = make_spec(model)
    out = np.zeros((D, D), dtype=np.complex128)
    _check(lib().qed_spec_hamiltonian(ctypes.byref(s), out.ctypes.data_as(_c_double_p), D * D),
           "qed_spec_hamiltonian")
    return out


def spec_jump(model, j):
    D, _ = spec_dim(model)
    s, _k = make_spec(model)
    out = np.zeros((D, D), dtype=np.complex128)
    _check(lib().qed_spec_jump(ctypes.byref(s), j, out.ctypes.data_as(_c_double_p), D * D), "qed_spec_jump")
    return out


def spec_restricted(model, keep, j=-1):
    """(P H P if j < 0 else P A_j P, d) on the basis states `keep` (host query of the
    operators qed_select_states builds)."""
    s, _k = make_spec(model)
    keep = np.ascontiguousarray(keep, dtype=np.int64)
    n = len(keep)
    out = np.zeros((n, n), dtype=np.complex128)
    d = np.zeros(n, dtype=np.float64)
    _check(lib().qed_spec_restricted(ctypes.byref(s), keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n,
                                     int(j), out.ctypes.data_as(_c_double_p), n * n, d.ctypes.data_as(_c_double_p)),
           "qed_spec_restricted")
    return out, d


def digit_positions(model):
    """Digit index of each cavity's photon number, each atom bit and each extra bit, in
    the layout documented in qed.h (per cavity: photon then atoms; extras last)."""
    photon, atom, pos = [], [], 0
    for c in range(model["n_cavities"]):
        photon.append(pos)
        pos += 1
        for _ in range(model["atoms_per_cavity"][c]):
            atom.append(pos)
            pos += 1
    extra = list(range(pos, pos + model["n_extra"]))
    return photon, atom, extra


def set_alloc_budget(nbytes):
    """Test hook (qed_set_alloc_budget): the library's device allocations fail with
    QED_ENOMEM once they would exceed `nbytes` in total; a negative value removes the limit."""
    _check(lib().qed_set_alloc_budget(int(nbytes)), "qed_set_alloc_budget")


def launch_count():
    """Kernels libqed has launched in this process."""
    n = ctypes.c_int64()
    _check(lib().qed_launch_count(ctypes.byref(n)), "qed_launch_count")
    return n.value


def tc_gemm(a_planes, b_planes, segments=((0, 0), (0, 1), (1, 0)), splits=1, stream=None):
    """Split-K partial sums [splits, M, N] (FP32) of sum over segments (p, q) of
    A_p B_q^T, the FP16 tensor-core product of the split-precision step; a_planes
    [planes, M, K] and b_planes [planes, N, K] are CUDA float16."""
    import torch
    M, N, K = _check_planes(a_planes, b_planes)
    seg = _arr([x for pq in segments for x in pq], np.int32)
    out = torch.empty((splits, M, N), dtype=torch.float32, device=a_planes.device)
    _check(lib().qed_tc_gemm(ctypes.c_void_p(a_planes.data_ptr()), a_planes.shape[0],
                             ctypes.c_void_p(b_planes.data_ptr()), b_planes.shape[0], M, N, K, len(segments),
                             seg.ctypes.data_as(_c_int32_p), splits, ctypes.c_void_p(out.data_ptr()),
                             _stream_handle(stream)), "qed_tc_gemm")
    return out


def tc_gemm_static(a_planes, b_planes, segments=((0, 0), (0, 1), (1, 0)), splits=1, out=None, stream=None):
    """The summed product [M, N] (FP32) of tc_gemm, computed without any device
    allocation inside the library: its split-K partials use the library's static scratch
    (splits * M * N <= 4 Mi floats).  `out` may be a caller-owned CUDA float32 tensor."""
    import torch
    M, N, K = _check_planes(a_planes, b_planes)
    seg = _arr([x for pq in segments for x in pq], np.int32)
    if out is None:
        out = torch.empty((M, N), dtype=torch.float32, device=a_planes.device)
    if (not isinstance(out, torch.Tensor) or out.dtype != torch.float32 or out.device != a_planes.device
            or tuple(out.shape) != (M, N) or not out.is_contiguous()):
        raise ValueError(f"out must be a contiguous float32 ({M}, {N}) tensor on {a_planes.device}")
    _check(lib().qed_tc_gemm_static(ctypes.c_void_p(a_planes.data_ptr()), a_planes.shape[0],
                                    ctypes.c_void_p(b_planes.data_ptr()), b_planes.shape[0], M, N, K,
                                    len(segments), seg.ctypes.data_as(_c_int32_p), splits,
                                    ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
           "qed_tc_gemm_static")
    return out


def _check_planes(a_planes, b_planes):
    """(M, N, K) of the FP16 operand stacks a_planes [planes, M, K] and b_planes [planes, N, K];
    both must be contiguous CUDA float16 tensors on one device with the same K (the library
    reads them through tensor maps encoded from these sizes)."""
    import torch
    for name, t in (("a_planes", a_planes), ("b_planes", b_planes)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float16 or not t.is_cuda or t.dim() != 3:
            raise TypeError(f"{name} must be a 3-d CUDA float16 tensor [planes, rows, K]")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if a_planes.device != b_planes.device:
        raise ValueError("a_planes and b_planes must be on one device")
    if a_planes.shape[2] != b_planes.shape[2]:
        raise ValueError(f"a_planes and b_planes must share K (got {a_planes.shape[2]} and {b_planes.shape[2]})")
    return a_planes.shape[1], b_planes.shape[1], a_planes.shape[2]


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Model:
    """A model built on the GPU: U = exp(-i H dt) and the operators, owned by libqed."""

    def __init__(self, model, precision="fp64", dt=None, stream=None, scheme="lie"):
        self.spec_dict = model
        self.precision = precision
        self.dt = float(model["dt"] if dt is None else dt)
        s, keep = make_spec(model)
        h = ctypes.c_void_p()
        _check(lib().qed_build(ctypes.byref(s), self.dt, PRECISIONS[precision], _stream_handle(stream),
                               ctypes.byref(h)), "qed_build")
        self._h = h
        d = ctypes.c_int64()
        _check(lib().qed_dim(self._h, ctypes.byref(d)), "qed_dim")
        self.dim = d.value
        n = ctypes.c_int32()
        _check(lib().qed_n_observables(self._h, ctypes.byref(n)), "qed_n_observables")
        self.n_observables = n.value
        self.n_digits = spec_dim(model)[1]
        self.scheme = "lie"
        if scheme != "lie":
            self.set_scheme(scheme)

    @classmethod
    def _from_handle(cls, h, parent):
        """Wraps a library-built model (e.g. one on a selected subset of parent's basis)."""
        self = cls.__new__(cls)
        self.spec_dict = parent.spec_dict
        self.precision = parent.precision
        self.dt = parent.dt
        self._h = h
        d = ctypes.c_int64()
        _check(lib().qed_dim(self._h, ctypes.byref(d)), "qed_dim")
        self.dim = d.value
        n = ctypes.c_int32()
        _check(lib().qed_n_observables(self._h, ctypes.byref(n)), "qed_n_observables")
        self.n_observables = n.value
        self.n_digits = parent.n_digits
        self.scheme = parent.scheme
        return self

    def close(self):
        if getattr(self, "_h", None):
            lib().qed_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def labels(self):
        out = np.zeros((self.dim, self.n_digits), dtype=np.int32)
        _check(lib().qed_basis_labels(self._h, out.ctypes.data_as(_c_int32_p)), "qed_basis_labels")
        return out

    def index_of(self, digits):
        d = _arr(digits, np.int32)
        idx = ctypes.c_int64()
        _check(lib().qed_basis_index(self._h, d.ctypes.data_as(_c_int32_p), ctypes.byref(idx)),
               "qed_basis_index")
        return idx.value

    def initial_index(self):
        """Index of the model's pure initial state (model['init'])."""
        photon, atom, extra = digit_positions(self.spec_dict)
        d = np.zeros(self.n_digits, dtype=np.int32)
        init = self.spec_dict["init"]
        for c, v in init.get("photons", {}).items():
            d[photon[int(c)]] = v
        for a, v in init.get("atoms", {}).items():
            d[atom[int(a)]] = v
        for x, v in init.get("extra", {}).items():
            d[extra[int(x)]] = v
        return self.index_of(d)

    def set_renorm_every(self, every):
        _check(lib().qed_set_renorm_every(self._h, int(every)), "qed_set_renorm_every")

    def set_plan(self, gemm1_bn, gemm1_splits, gemm2_bn, gemm2_splits, stream=None):
        """Sets the tile widths and split-K factors of the step's two products (qed_set_plan)."""
        _check(lib().qed_set_plan(self._h, int(gemm1_bn), int(gemm1_splits), int(gemm2_bn), int(gemm2_splits),
                                  _stream_handle(stream)), "qed_set_plan")

    def autotune(self, steps=20, stream=None):
        """Times the step's tile widths and split-K factors (qed_autotune) and keeps the
        fastest; returns the description of the choice."""
        buf = ctypes.create_string_buffer(256)
        _check(lib().qed_autotune(self._h, int(steps), buf, 256, _stream_handle(stream)), "qed_autotune")
        return buf.value.decode()

    def set_wait_gate(self, closed, budget_cycles=100000, stream=None):
        """Test hook (qed_set_wait_gate): while closed, the split step's tensor-core kernels
        time out on a bounded wait before doing any work, and sync() raises QED_ETIMEOUT."""
        _check(lib().qed_set_wait_gate(self._h, 1 if closed else 0, int(budget_cycles), _stream_handle(stream)),
               "qed_set_wait_gate")

    def set_scheme(self, scheme):
        """'lie' (first order), 'strang' (second order: half Lindblad steps by the explicit
        midpoint rule around the unitary) or 'effective' (the anticommutator inside a
        non-unitary propagator, then the jump terms)."""
        _check(lib().qed_set_scheme(self._h, SCHEMES[scheme]), "qed_set_scheme")
        self.scheme = scheme

    @staticmethod
    def n_records(n_steps, record_every, step_offset=0):
        if record_every <= 0:
            return 0
        return sum(1 for i in range(n_steps + 1) if (step_offset + i) % record_every == 0)

    def evolve(self, rho, n_steps, record_every=0, obs_ids=None, records=None, step_offset=0, stream=None):
        """Advance rho (CUDA complex128 D x D tensor) in place; returns the records tensor."""
        import torch
        _check_rho(rho, self.dim)
        ids = _arr(obs_ids if obs_ids is not None else [], np.int32)
        n_obs = 0 if obs_ids is None else len(obs_ids)
        if n_obs and records is None:
            nrec = self.n_records(n_steps, record_every, step_offset)
            records = torch.zeros((nrec, n_obs), dtype=torch.float64, device=rho.device)
        rec_ptr = ctypes.c_void_p(records.data_ptr()) if records is not None else ctypes.c_void_p()
        _check(lib().qed_evolve(self._h, ctypes.c_void_p(rho.data_ptr()), int(n_steps), int(step_offset),
                                int(record_every), n_obs, ids.ctypes.data_as(_c_int32_p), rec_ptr,
                                _stream_handle(stream)), "qed_evolve")
        return records

    def observables(self, rho, obs_ids, out=None, stream=None):
        import torch
        _check_rho(rho, self.dim)
        ids = _arr(obs_ids, np.int32)
        if out is None:
            out = torch.zeros(len(obs_ids), dtype=torch.float64, device=rho.device)
        _check(lib().qed_observables(self._h, ctypes.c_void_p(rho.data_ptr()), len(obs_ids),
                                     ids.ctypes.data_as(_c_int32_p), ctypes.c_void_p(out.data_ptr()),
                                     _stream_handle(stream)), "qed_observables")
        return out

    def adjoint(self, rho0, n_steps, obs_diag, checkpoint_every=50, stream=None):
        """(loss, grad_g, grad_zeta, grad_gamma) of tr(diag(obs_diag) rho_N) as CUDA FP64
        tensors; rho0 a CUDA complex128 D x D tensor, obs_diag a CUDA FP64 vector."""
        import torch
        _check_rho(rho0, self.dim)
        m = self.spec_dict
        dev = rho0.device
        loss = torch.zeros(1, dtype=torch.float64, device=dev)
        gg = torch.zeros(max(len(m["g"]), 1), dtype=torch.float64, device=dev)
        gz = torch.zeros(max(len(m["zeta"]), 1), dtype=torch.float64, device=dev)
        gj = torch.zeros(max(len(m["jumps"]), 1), dtype=torch.float64, device=dev)
        o = obs_diag.to(device=dev, dtype=torch.float64).contiguous()
        _check(lib().qed_adjoint(self._h, ctypes.c_void_p(rho0.data_ptr()), int(n_steps), int(checkpoint_every),
                                 ctypes.c_void_p(o.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                 ctypes.c_void_p(gg.data_ptr()), ctypes.c_void_p(gz.data_ptr()),
                                 ctypes.c_void_p(gj.data_ptr()), _stream_handle(stream)), "qed_adjoint")
        return loss[0], gg[: len(m["g"])], gz[: len(m["zeta"])], gj[: len(m["jumps"])]

    def sync(self, stream=None):
        _check(lib().qed_sync_status(self._h, _stream_handle(stream)), "qed_sync_status")

    def set_U(self, U, stream=None):
        _check_rho(U, self.dim)
        _check(lib().qed_set_U(self._h, ctypes.c_void_p(U.data_ptr()), _stream_handle(stream)), "qed_set_U")

    def get_U(self, stream=None):
        import torch
        U = torch.empty((self.dim, self.dim), dtype=torch.complex128, device="cuda")
        _check(lib().qed_get_U(self._h, ctypes.c_void_p(U.data_ptr()), _stream_handle(stream)), "qed_get_U")
        return U

    def profile(self, rho, n_steps, stream=None):
        """Mean milliseconds per step of each kernel class (CUDA events on the stream)."""
        _check_rho(rho, self.dim)
        ms = np.zeros(8, dtype=np.float64)
        names = ctypes.create_string_buffer(512)
        _check(lib().qed_profile(self._h, ctypes.c_void_p(rho.data_ptr()), int(n_steps),
                                 ms.ctypes.data_as(_c_double_p), 8, names, 512, _stream_handle(stream)),
               "qed_profile")
        labels = [x for x in names.value.decode().split(",") if x]
        return dict(zip(labels, ms[: len(labels)].tolist()))

    def profile_replay(self, rho, reps=200, stream=None):
        """Mean milliseconds per launch of each kernel of the split Lie step, every kernel
        replayed back to back from a CUDA graph (qed_profile_replay)."""
        return _profile_replay(self, rho, reps, stream)


def _profile_replay(model, rho, reps, stream=None):
    _check_rho(rho, model.dim)
    ms = np.zeros(8, dtype=np.float64)
    names = ctypes.create_string_buffer(512)
    _check(lib().qed_profile_replay(model._h, ctypes.c_void_p(rho.data_ptr()), int(reps),
                                    ms.ctypes.data_as(_c_double_p), 8, names, 512, _stream_handle(stream)),
           "qed_profile_replay")
    labels = [x for x in names.value.decode().split(",") if x]
    return dict(zip(labels, ms[: len(labels)].tolist()))


def evolve_batched(models, rhos, n_steps, record_every=0, records=None, stream=None):
    """Advance every rhos[i] (CUDA complex128, in place) by n_steps steps of models[i]
    together (qed_evolve_batched).  With record_every > 0 returns, per instance, a CUDA
    FP64 tensor [n_rec, D_i] of populations (or fills the given `records` tensors)."""
    import torch
    n = len(models)
    if n != len(rhos):
        raise ValueError("one rho per model")
    for m, r in zip(models, rhos):
        _check_rho(r, m.dim)
    if record_every > 0 and records is None:
        nrec = n_steps // record_every + 1
        records = [torch.zeros((nrec, m.dim), dtype=torch.float64, device=r.device) for m, r in zip(models, rhos)]
    H = (ctypes.c_void_p * n)(*[m._h.value for m in models])
    R = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rhos])
    rec = None
    if records is not None:
        rec = (ctypes.c_void_p * n)(*[x.data_ptr() for x in records])
    _check(lib().qed_evolve_batched(n, H, R, int(n_steps), int(record_every), rec, _stream_handle(stream)),
           "qed_evolve_batched")
    return records


def autotune_batched(models, steps=3, stream=None):
    """Times the GEMM1 tile widths of the grouped launches on whole batched steps of these
    models (qed_autotune_batched) and keeps the fastest in them; returns the description."""
    n = len(models)
    H = (ctypes.c_void_p * n)(*[m._h.value for m in models])
    buf = ctypes.create_string_buffer(256)
    _check(lib().qed_autotune_batched(n, H, int(steps), buf, 256, _stream_handle(stream)), "qed_autotune_batched")
    return buf.value.decode()


def select_states(model, rho0, steps_per_round, n_rounds, eps, stream=None):
    """State space selection (qed_select_states): rounds of solving, deleting the states
    whose probability grows slower than eps, and normalising.  Returns (Model on the kept
    states, its density matrix as a CUDA complex128 tensor, kept indices in model's basis,
    dimension after each round)."""
    import torch
    _check_rho(rho0, model.dim)
    D = model.dim
    out = torch.zeros(D * D, dtype=torch.complex128, device=rho0.device)
    keep = np.zeros(D, dtype=np.int64)
    sizes = np.zeros(n_rounds, dtype=np.int64)
    n = ctypes.c_int64()
    h = ctypes.c_void_p()
    _check(lib().qed_select_states(model._h, ctypes.c_void_p(rho0.data_ptr()), int(steps_per_round), int(n_rounds),
                                   float(eps), ctypes.byref(h), ctypes.c_void_p(out.data_ptr()),
                                   keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(n),
                                   sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _stream_handle(stream)),
           "qed_select_states")
    k = n.value
    reduced = Model._from_handle(h, model)
    return reduced, out[:k * k].view(k, k).clone(), keep[:k].copy(), sizes


def _check_rho(rho, dim):
    import torch
    if not isinstance(rho, torch.Tensor) or rho.dtype != torch.complex128 or not rho.is_cuda:
        raise TypeError("expected a CUDA complex128 tensor")
    if tuple(rho.shape) != (dim, dim) or not rho.is_contiguous():
        raise ValueError(f"expected a contiguous {dim} x {dim} tensor")


def _autograd_function():
    import torch

    class QMELoss(torch.autograd.Function):
        """L = tr(diag(obs) rho_N) as a differentiable function of the couplings g, the
        hoppings zeta and the rates gamma (CPU or CUDA FP64 tensors).  The forward builds
        the model with these parameters and runs qed_adjoint, whose gradients the backward
        returns (scaled by the incoming gradient)."""

        @staticmethod
        def forward(ctx, g, zeta, gamma, model, rho0, n_steps, obs_diag, checkpoint_every, precision):
            m = dict(model)
            m["g"] = [float(x) for x in g.detach().cpu()]
            m["zeta"] = [float(x) for x in zeta.detach().cpu()]
            m["jumps"] = [(k, s_, float(x)) for (k, s_, _), x in zip(model["jumps"], gamma.detach().cpu())]
            gm = Model(m, precision=precision)
            loss, gg, gz, gj = gm.adjoint(rho0, n_steps, obs_diag, checkpoint_every)
            ctx.save_for_backward(gg.to(g.device), gz.to(zeta.device), gj.to(gamma.device))
            gm.close()
            return loss.to(g.device)

        @staticmethod
        def backward(ctx, grad_out):
            gg, gz, gj = ctx.saved_tensors
            return grad_out * gg, grad_out * gz, grad_out * gj, None, None, None, None, None, None

    return QMELoss


def fit_final_populations(*args, **kwargs):
    """Least-squares fit of couplings to final populations (see fit.fit_final_populations)."""
    from . import fit
    return fit.fit_final_populations(*args, **kwargs)


def qme_loss(g, zeta, gamma, model, rho0, n_steps, obs_diag, checkpoint_every=50, precision="fp64"):
    """Differentiable tr(diag(obs_diag) rho_N) (see QMELoss)."""
    return _autograd_function().apply(g, zeta, gamma, model, rho0, n_steps, obs_diag, checkpoint_every,
                                      precision)
