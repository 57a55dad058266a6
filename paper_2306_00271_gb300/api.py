"""Python binding of libtrheed (include/trheed.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels. PyTorch provides device memory
(tensors' data pointers) and the current CUDA stream. Loading fails loudly when the library is
missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtrheed.so")
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "trheed.h")

TRH_OK, TRH_EINVAL, TRH_EGRAZING, TRH_ESINGULAR = 0, -1, -2, -3
TRH_ETIMEOUT, TRH_ENOMEM, TRH_ECUDA, TRH_EUNSUPPORTED, TRH_ENOCONV = -4, -5, -6, -7, -8
INTEGRATORS = {"sp4": 0, "sp6": 1, "rk4": 2, "conventional": 3}
PRECISIONS = {"fp64": 0, "mixed": 1}
SPLIT_MODES = {"auto": 0, "off": 1, "on": 2}


class TrhProblem(C.Structure):
    _fields_ = [
        ("particle", C.c_int), ("energy_ev", C.c_double), ("absorption", C.c_double),
        ("a1", C.c_double * 2), ("a2", C.c_double * 2),
        ("n_beams", C.c_int), ("beams", C.POINTER(C.c_int)),
        ("n_atoms", C.c_int), ("atoms", C.POINTER(C.c_double)), ("dw", C.POINTER(C.c_double)),
        ("species", C.POINTER(C.c_int)), ("n_species", C.c_int), ("sf", C.POINTER(C.c_double)),
        ("z_e", C.c_double), ("n_steps", C.c_int), ("integrator", C.c_int),
        ("rhst_threshold", C.c_double), ("precision", C.c_int),
    ]


class TrhStats(C.Structure):
    _fields_ = [
        ("n_sets", C.c_int), ("n_angles", C.c_int), ("n_beams", C.c_int), ("n_nodes", C.c_int),
        ("rhst_total", C.c_longlong), ("rhst_max", C.c_int), ("n_bad", C.c_int),
        ("first_bad_set", C.c_int), ("first_bad_angle", C.c_int), ("first_bad_status", C.c_int),
        ("kernels_launched", C.c_int), ("ms_last", C.c_double),
        ("ms_potential", C.c_double), ("ms_integrate", C.c_double),
        ("ms_gradient", C.c_double), ("wide_tile", C.c_int), ("graph_replay", C.c_int),
        ("bulk_periods", C.c_int), ("ms_bulk", C.c_double), ("column_split", C.c_int),
        ("ctas_per_pair", C.c_int), ("set_chunks", C.c_int), ("tuned", C.c_int),
        ("sweep_split", C.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TrhError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"trheed error {code}: {msg}")
        self.code = code


_lib = None


def header_functions():
    """Names of the functions include/trheed.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(trh_[a-z_]+)\s*\(", txt)))


def load():
    """Load libtrheed.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2306_00271_gb300.build` (no CPU fallback exists)")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    lib.trh_create.argtypes = [C.POINTER(vp), C.POINTER(TrhProblem)]
    lib.trh_set_structure.argtypes = [vp, C.c_int, vp, vp]
    lib.trh_rocking_curve.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp]
    lib.trh_query.argtypes = [vp, C.POINTER(TrhStats)]
    lib.trh_strerror.argtypes = [C.c_int]
    lib.trh_strerror.restype = C.c_char_p
    lib.trh_last_error.restype = C.c_char_p
    lib.trh_destroy.argtypes = [vp]
    lib.trh_destroy.restype = None
    lib.trh_rocking_curve_noalloc.argtypes = [C.POINTER(TrhProblem), C.c_int, vp, vp, vp, vp, vp]
    lib.trh_rocking_curve_noalloc.restype = C.c_int
    lib.trh_set_fit.argtypes = [vp, C.c_int, vp, C.c_int, vp, C.c_int]
    lib.trh_set_bulk.argtypes = [vp, C.c_int, vp, vp, vp, C.c_double, C.c_int, C.c_int,
                                 C.c_double]
    lib.trh_set_column_split.argtypes = [vp, C.c_int]
    lib.trh_set_async.argtypes = [vp, C.c_int]
    lib.trh_set_image_budget.argtypes = [vp, C.c_size_t]
    lib.trh_curve_jacobian.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp]
    lib.trh_rfactor_grad.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp, vp]
    lib.trh_batch_create.argtypes = [C.POINTER(vp)]
    lib.trh_batch_add.argtypes = [vp, vp, C.c_int, vp, vp, vp, vp]
    lib.trh_batch_run.argtypes = [vp, vp]
    lib.trh_batch_query.argtypes = [vp, C.POINTER(TrhStats)]
    lib.trh_batch_destroy.argtypes = [vp]
    lib.trh_batch_destroy.restype = None
    for f in ("trh_create", "trh_set_structure", "trh_rocking_curve", "trh_query", "trh_set_fit",
              "trh_curve_jacobian", "trh_rfactor_grad", "trh_set_bulk", "trh_set_column_split", "trh_set_async",
              "trh_set_image_budget",
              "trh_batch_create",
              "trh_batch_add",
              "trh_batch_run", "trh_batch_query"):
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


def _check(code: int):
    if code != TRH_OK:
        lib = load()
        raise TrhError(code, lib.trh_last_error().decode())


def _ptr(a) -> C.c_void_p:
    if a is None:
        return C.c_void_p(0)
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def make_problem(wl, precision: str = "fp64", integrator: str = "sp4",
                 threshold: float = 1000.0):
    """(TrhProblem, arrays it points into) for a workload; keep the arrays alive with it."""
    keep = dict(
        beams=np.ascontiguousarray(wl.beams, dtype=np.int32),
        atoms=np.ascontiguousarray(wl.atoms, dtype=np.float64),
        dw=np.ascontiguousarray(wl.dw, dtype=np.float64),
        species=np.ascontiguousarray(wl.species, dtype=np.int32),
        sf=np.ascontiguousarray(wl.sf, dtype=np.float64))
    p = TrhProblem()
    p.particle = int(wl.particle)
    p.energy_ev = float(wl.energy_ev)
    p.absorption = float(wl.absorption)
    p.a1[0], p.a1[1] = float(wl.a1[0]), float(wl.a1[1])
    p.a2[0], p.a2[1] = float(wl.a2[0]), float(wl.a2[1])
    p.n_beams = int(keep["beams"].shape[0])
    p.beams = keep["beams"].ctypes.data_as(C.POINTER(C.c_int))
    p.n_atoms = int(keep["atoms"].shape[0])
    p.atoms = keep["atoms"].ctypes.data_as(C.POINTER(C.c_double))
    p.dw = keep["dw"].ctypes.data_as(C.POINTER(C.c_double))
    p.species = keep["species"].ctypes.data_as(C.POINTER(C.c_int))
    p.n_species = int(keep["sf"].shape[0])
    p.sf = keep["sf"].ctypes.data_as(C.POINTER(C.c_double))
    p.z_e = float(wl.z_e)
    p.n_steps = int(wl.n_steps)
    p.integrator = INTEGRATORS[integrator]
    p.rhst_threshold = float(threshold)
    p.precision = PRECISIONS[precision]
    return p, keep


def rocking_curve_noalloc(wl, theta0, theta1, rho, eta, integrator: str = "sp4",
                          threshold: float = 1000.0, stream=None):
    """trh_rocking_curve_noalloc: binary64 curve of one structure using only the library's fixed
    device array (no device allocation). theta0/theta1 (A,) float64, rho (A, N) complex128 and
    eta (A, N) float64 must be CUDA tensors; the work is enqueued on `stream` (default: torch's
    current stream) and not synchronised."""
    lib = load()
    p, keep = make_problem(wl, "fp64", integrator, threshold)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib.trh_rocking_curve_noalloc(C.byref(p), int(theta0.numel()), _ptr(theta0),
                                         _ptr(theta1), _ptr(rho), _ptr(eta), C.c_void_p(stream)))
    return rho, eta


class Engine:
    """One context of libtrheed: a beam set, slab, integrator and precision, and one or more
    parameter sets (structures)."""

    def __init__(self, wl, precision: str = "fp64", integrator: str = "sp4",
                 threshold: float = 1000.0):
        self.lib = load()
        self.wl = wl
        self.N = int(wl.beams.shape[0])
        self._keep = dict(
            beams=np.ascontiguousarray(wl.beams, dtype=np.int32),
            atoms=np.ascontiguousarray(wl.atoms, dtype=np.float64),
            dw=np.ascontiguousarray(wl.dw, dtype=np.float64),
            species=np.ascontiguousarray(wl.species, dtype=np.int32),
            sf=np.ascontiguousarray(wl.sf, dtype=np.float64))
        k = self._keep
        p = TrhProblem()
        p.particle = int(wl.particle)
        p.energy_ev = float(wl.energy_ev)
        p.absorption = float(wl.absorption)
        p.a1[0], p.a1[1] = float(wl.a1[0]), float(wl.a1[1])
        p.a2[0], p.a2[1] = float(wl.a2[0]), float(wl.a2[1])
        p.n_beams = self.N
        p.beams = k["beams"].ctypes.data_as(C.POINTER(C.c_int))
        p.n_atoms = int(k["atoms"].shape[0])
        p.atoms = k["atoms"].ctypes.data_as(C.POINTER(C.c_double))
        p.dw = k["dw"].ctypes.data_as(C.POINTER(C.c_double))
        p.species = k["species"].ctypes.data_as(C.POINTER(C.c_int))
        p.n_species = int(k["sf"].shape[0])
        p.sf = k["sf"].ctypes.data_as(C.POINTER(C.c_double))
        p.z_e = float(wl.z_e)
        p.n_steps = int(wl.n_steps)
        p.integrator = INTEGRATORS[integrator]
        p.rhst_threshold = float(threshold)
        p.precision = PRECISIONS[precision]
        self.n_atoms = p.n_atoms
        self.n_sets = 1
        self.ctx = C.c_void_p()
        _check(self.lib.trh_create(C.byref(self.ctx), C.byref(p)))

    def set_structures(self, atoms, dw=None):
        """atoms (n_sets, n_atoms, 3) and dw (n_sets, n_atoms): numpy arrays, or CUDA float64
        tensors (copied on the device; no host round trip)."""
        if hasattr(atoms, "is_cuda") and atoms.is_cuda:
            a = atoms.contiguous()
            d = None if dw is None else dw.contiguous()
            n_sets = a.numel() // (3 * self.n_atoms)
            _check(self.lib.trh_set_structure(self.ctx, n_sets, _ptr(a), _ptr(d)))
            self.n_sets = n_sets
            return
        atoms = np.ascontiguousarray(atoms, dtype=np.float64).reshape(-1, self.n_atoms, 3)
        dwp = None if dw is None else np.ascontiguousarray(dw, dtype=np.float64).reshape(
            atoms.shape[0], self.n_atoms)
        _check(self.lib.trh_set_structure(self.ctx, atoms.shape[0], _ptr(atoms), _ptr(dwp)))
        self.n_sets = atoms.shape[0]

    def rocking_curve(self, theta0, theta1=None, rho=None, eta=None, stream=None):
        """Device path: theta0/theta1 torch float64 tensors (any device) or arrays; returns
        (rho, eta) as torch tensors on the current CUDA device, shape (n_sets, A, N)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        t0 = torch.as_tensor(theta0, dtype=torch.float64).to(dev).contiguous()
        t1 = (torch.full_like(t0, float(self.wl.theta1[0])) if theta1 is None
              else torch.as_tensor(theta1, dtype=torch.float64).to(dev).contiguous())
        A = t0.numel()
        if rho is None:
            rho = torch.empty((self.n_sets, A, self.N), dtype=torch.complex128, device=dev)
        if eta is None:
            eta = torch.empty((self.n_sets, A, self.N), dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(self.lib.trh_rocking_curve(self.ctx, A, _ptr(t0), _ptr(t1), _ptr(rho), _ptr(eta),
                                          C.c_void_p(st)))
        return rho, eta

    def rocking_curve_host(self, theta0, theta1=None, rho=None, eta=None, stream=None):
        """Host path: numpy (or pinned torch) inputs and outputs; the library copies."""
        t0 = np.ascontiguousarray(np.atleast_1d(theta0), dtype=np.float64)
        t1 = (np.full_like(t0, float(self.wl.theta1[0])) if theta1 is None
              else np.ascontiguousarray(np.atleast_1d(theta1), dtype=np.float64))
        A = t0.size
        if rho is None:
            rho = np.empty((self.n_sets, A, self.N), dtype=np.complex128)
        if eta is None:
            eta = np.empty((self.n_sets, A, self.N), dtype=np.float64)
        _check(self.lib.trh_rocking_curve(self.ctx, A, _ptr(t0), _ptr(t1), _ptr(rho), _ptr(eta),
                                          C.c_void_p(0 if stream is None else stream)))
        return rho, eta

    def set_bulk(self, atoms, dw, species, period: float, steps_per_period: int,
                 max_periods: int = 500, tol: float = 1e-12):
        """Ideal bulk below z_e (one period's atoms, z relative to the period top in (-d, 0]);
        slab integrations then start from the converged bulk boundary condition."""
        a = np.ascontiguousarray(atoms, dtype=np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(dw, dtype=np.float64).reshape(-1)
        sp = np.ascontiguousarray(species, dtype=np.int32).reshape(-1)
        self._bulk = (a, d, sp)
        _check(self.lib.trh_set_bulk(self.ctx, a.shape[0], _ptr(a), _ptr(d), _ptr(sp),
                                     float(period), int(steps_per_period), int(max_periods),
                                     float(tol)))

    def set_column_split(self, mode: str = "auto"):
        """Mixed and FP64 (N <= 64) paths: two CTAs per (set, angle) pair ("on"), one ("off"),
        or two when the call's pairs fit on half the SMs ("auto", the default). Results are
        identical."""
        _check(self.lib.trh_set_column_split(self.ctx, SPLIT_MODES[mode]))

    def set_async(self, on: bool = True):
        """Calls return once their work is enqueued; stats() waits for the last call and
        completes its per-pair counters (a failing pair shows there, not as an exception)."""
        _check(self.lib.trh_set_async(self.ctx, 1 if on else 0))

    def set_image_budget(self, nbytes: int = 0):
        """Mixed path: device bytes of digit images kept at once (0: the default, 40 GiB); sets
        beyond it run in chunks (stats()["set_chunks"]). Results do not depend on it."""
        _check(self.lib.trh_set_image_budget(self.ctx, int(nbytes)))

    def set_fit(self, free_atoms, dw_class=None, ckpt_every: int = 64):
        """Fit parameters for curve_jacobian / rfactor_grad: z of the atoms ``free_atoms`` and
        one B per Debye-Waller class (``dw_class[a]`` = class of atom a, -1 = fixed B)."""
        fa = np.ascontiguousarray(free_atoms, dtype=np.int32).reshape(-1)
        if dw_class is None:
            cls, n_classes = None, 0
        else:
            cls = np.ascontiguousarray(dw_class, dtype=np.int32).reshape(-1)
            n_classes = int(cls.max()) + 1 if cls.size and cls.max() >= 0 else 0
        self._fit = (fa, cls)
        _check(self.lib.trh_set_fit(self.ctx, int(fa.size), _ptr(fa), n_classes, _ptr(cls),
                                    int(ckpt_every)))
        self.n_free, self.n_classes = int(fa.size), n_classes

    def _angles(self, theta0, theta1, dev):
        import torch
        t0 = torch.as_tensor(theta0, dtype=torch.float64).to(dev).contiguous()
        t1 = (torch.full_like(t0, float(self.wl.theta1[0])) if theta1 is None
              else torch.as_tensor(theta1, dtype=torch.float64).to(dev).contiguous())
        return t0, t1

    def curve_jacobian(self, theta0, theta1=None, stream=None):
        """(eta (n_sets, A, N), jac (n_sets, A, n_free + n_classes)) as CUDA tensors:
        d eta_1 / d z of the free atoms, then d eta_1 / d B of the classes (reverse sweep)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        t0, t1 = self._angles(theta0, theta1, dev)
        A = t0.numel()
        eta = torch.empty((self.n_sets, A, self.N), dtype=torch.float64, device=dev)
        jac = torch.empty((self.n_sets, A, self.n_free + self.n_classes), dtype=torch.float64,
                          device=dev)
        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(self.lib.trh_curve_jacobian(self.ctx, A, _ptr(t0), _ptr(t1), _ptr(eta), _ptr(jac),
                                           C.c_void_p(st)))
        return eta, jac

    def rfactor_grad(self, theta0, theta1, target, stream=None):
        """(R (n_sets,), dR/dz (n_sets, n_free), dR/dB (n_sets, n_classes)) as CUDA tensors."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        t0, t1 = self._angles(theta0, theta1, dev)
        tg = torch.as_tensor(target, dtype=torch.float64).to(dev).contiguous()
        R = torch.empty(self.n_sets, dtype=torch.float64, device=dev)
        gz = torch.empty((self.n_sets, self.n_free), dtype=torch.float64, device=dev)
        gb = torch.empty((self.n_sets, self.n_classes), dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(self.lib.trh_rfactor_grad(self.ctx, t0.numel(), _ptr(t0), _ptr(t1), _ptr(tg),
                                         _ptr(R), _ptr(gz), _ptr(gb), C.c_void_p(st)))
        return R, gz, gb

    def stats(self) -> dict:
        s = TrhStats()
        _check(self.lib.trh_query(self.ctx, C.byref(s)))
        return s.as_dict()

    def close(self):
        if self.ctx:
            self.lib.trh_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Rocking curves of several engines (any beam counts) in persistent launches replayed from a
    CUDA graph (trh_batch_*). Angles and outputs are CUDA tensors owned by the batch."""

    def __init__(self):
        self.lib = load()
        self.h = C.c_void_p()
        _check(self.lib.trh_batch_create(C.byref(self.h)))
        self.jobs = []

    def add(self, engine: "Engine", theta0, theta1=None):
        """Queue all parameter sets of ``engine`` at the given angles; returns (rho, eta) CUDA
        tensors (n_sets, A, N) that every run() overwrites."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        t0, t1 = engine._angles(theta0, theta1, dev)
        A = t0.numel()
        rho = torch.empty((engine.n_sets, A, engine.N), dtype=torch.complex128, device=dev)
        eta = torch.empty((engine.n_sets, A, engine.N), dtype=torch.float64, device=dev)
        _check(self.lib.trh_batch_add(self.h, engine.ctx, A, _ptr(t0), _ptr(t1), _ptr(rho),
                                      _ptr(eta)))
        self.jobs.append((engine, t0, t1, rho, eta))
        return rho, eta

    def run(self, stream=None):
        import torch
        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(self.lib.trh_batch_run(self.h, C.c_void_p(st)))

    def stats(self) -> dict:
        s = TrhStats()
        _check(self.lib.trh_batch_query(self.h, C.byref(s)))
        return s.as_dict()

    def close(self):
        if self.h:
            self.lib.trh_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rfactor_function():
    import torch

    class RFactorFunction(torch.autograd.Function):
        """R(z, B) of a fit with its gradient from the library's reverse sweep."""

        @staticmethod
        def forward(ctx, z, b, fit):
            R, gz, gb = fit._evaluate(z, b)
            ctx.save_for_backward(gz, gb)
            return R

        @staticmethod
        def backward(ctx, gR):
            gz, gb = ctx.saved_tensors
            return gR[:, None] * gz, gR[:, None] * gb, None

    return RFactorFunction


class RFactor:
    """The reverse-analysis objective (Section 1: argmin over structures of the misfit between
    measured and computed curves) as a differentiable torch function.

    ``fit(z, b)`` takes z (n_sets, n_free) coordinates of the free atoms and b (n_sets,
    n_classes) Debye-Waller factors of the classes (CUDA float64 tensors), writes them into the
    structure, and returns R (n_sets,) whose backward pass uses the adjoint gradients computed
    in the same library call (no extra forward run)."""

    def __init__(self, engine: "Engine", free_atoms, dw_class, theta0, theta1, target,
                 ckpt_every: int = 64):
        import torch
        self.engine = engine
        engine.set_fit(free_atoms, dw_class, ckpt_every)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.free = torch.as_tensor(np.asarray(free_atoms, dtype=np.int64), device=dev)
        cls = np.asarray(dw_class, dtype=np.int64)
        self.members = torch.as_tensor(np.nonzero(cls >= 0)[0], device=dev)
        self.member_class = torch.as_tensor(cls[cls >= 0], device=dev)
        self.atoms0 = torch.as_tensor(np.asarray(engine.wl.atoms, dtype=np.float64), device=dev)
        self.dw0 = torch.as_tensor(np.asarray(engine.wl.dw, dtype=np.float64), device=dev)
        self.theta0, self.theta1, self.target = theta0, theta1, target
        self._fn = _rfactor_function()

    def _evaluate(self, z, b):
        n_sets = z.shape[0]
        atoms = self.atoms0.expand(n_sets, -1, -1).clone()
        atoms[:, self.free, 2] = z.detach()
        dw = self.dw0.expand(n_sets, -1).clone()
        dw[:, self.members] = b.detach()[:, self.member_class]
        self.engine.set_structures(atoms.contiguous(), dw.contiguous())
        return self.engine.rfactor_grad(self.theta0, self.theta1, self.target)

    def __call__(self, z, b):
        return self._fn.apply(z, b, self)
