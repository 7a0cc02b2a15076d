"""Python binding of the single-image FCM entry points (argument marshalling only).

Every step of the computation runs in the CUDA library; this module only
turns torch tensors or numpy arrays into pointers, picks the current torch
stream, and turns status codes into exceptions.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import _lib


_SLICE_DTYPE = np.dtype(_lib.fcm_slice)


def _ptr(a) -> int:
    """Device or host pointer of a contiguous float32 torch tensor / numpy array."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy arrays must be C-contiguous float32")
        return a.ctypes.data
    import torch
    if not isinstance(a, torch.Tensor):
        raise TypeError(f"expected a torch tensor or numpy array, got {type(a)}")
    if a.dtype != torch.float32 or not a.is_contiguous():
        raise TypeError("tensors must be contiguous float32")
    return a.data_ptr()


def _numel(a) -> int:
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


@dataclass
class FCMResult:
    U: object
    V: object
    iters: int
    status: int
    delta: float
    J: float
    V64: np.ndarray
    flags: int
    launches: int = 0
    trace: dict | None = field(default=None)

    @property
    def converged(self) -> bool:
        return self.status == _lib.FCM_OK


@dataclass
class Slice:
    """One image of a batch. ``x`` is a CUDA float32 tensor of n pixels; give
    ``U0`` [C, n] (read only) or ``V0`` (C initial centers). ``U`` and ``V``
    receive the results (allocated when None). After the run the result
    fields are filled."""
    x: object
    C: int
    m: float = 2.0
    eps: float = 1e-5
    max_iter: int = 300
    U0: object = None
    V0: object = None
    U: object = None
    V: object = None
    iters: int = 0
    status: int = 0
    flags: int = 0
    delta: float = 0.0
    J: float = 0.0
    V64: np.ndarray | None = None
    init: str = ""           # start the last run took: "U" (U0) or "V" (centers)
    V0_warm: np.ndarray | None = None  # predicted centers a warm-started run began from


class Batch:
    """Slices marshalled once into the library's fcm_slice array, for batches
    run again and again on the same buffers (a serving loop, a benchmark).
    Pass it wherever a list of slices is taken; the slices' result fields are
    filled after each run as usual."""

    def __init__(self, slices):
        self.slices = list(slices)
        self.arr = FCM._c_slices(self.slices)
        self._init = self.arr[["init_mode", "V0"]].copy()

    def reset(self):
        """Back to each slice's own start (a warm-started run rewrites it)."""
        self.arr["init_mode"] = self._init["init_mode"]
        self.arr["V0"] = self._init["V0"]

    def read_back(self):
        """Copy the last run's per-slice results from ``arr`` into the Slice
        fields (iters, status, flags, delta, J, V64, init, V0_warm)."""
        FCM._read_back(self.arr, self.slices)

    def __len__(self):
        return len(self.slices)


def _as_batch(slices) -> Batch:
    if isinstance(slices, Batch):
        slices.reset()
        return slices
    return Batch(slices)


class FCM:
    """A handle of the CUDA FCM library bound to one device.

    Work is issued on torch's current CUDA stream of that device at each call.
    """

    def __init__(self, device: int | None = None):
        import torch
        self._lib = _lib.load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._h = ctypes.c_void_p()
        _lib.check(self._lib.fcm_create(ctypes.byref(self._h), self.device, None))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.fcm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_limits(self, grid_wait_spins: int = 0, tma_wait_polls: int = 0, barrier_phantoms: int = 0,
                   fail_alloc_in: int = 0, defaults: bool = False):
        """Bounds of the device-side waits and test-only fault injection
        (fcm_set_limits); ``defaults=True`` restores every default."""
        if defaults:
            _lib.check(self._lib.fcm_set_limits(self._h, None), self._h)
            return
        lim = _lib.fcm_limits(grid_wait_spins, tma_wait_polls, barrier_phantoms, fail_alloc_in)
        _lib.check(self._lib.fcm_set_limits(self._h, ctypes.byref(lim)), self._h)

    def limits(self) -> dict:
        lim = _lib.fcm_limits()
        _lib.check(self._lib.fcm_get_limits(self._h, ctypes.byref(lim)), self._h)
        return {k: getattr(lim, k) for k, _ in lim._fields_}

    def _bind_stream(self):
        import torch
        s = torch.cuda.current_stream(self.device).cuda_stream
        _lib.check(self._lib.fcm_set_stream(self._h, ctypes.c_void_p(s)), self._h)

    def run(self, x, C: int, m: float = 2.0, eps: float = 1e-5, max_iter: int = 300, *,
            U0=None, V0=None, U=None, V=None, trace: bool = False, graph: bool = True,
            tma: bool = True, persistent: bool = True, recompute: bool = False,
            deterministic: bool = False, raise_on_error: bool = True) -> FCMResult:
        """Algorithm 1 on one image.

        ``x``: n float32 pixels (CUDA tensor, pinned/CPU tensor or numpy).
        Start from memberships: ``U0`` [C, n] (read only), or no ``U0`` and
        ``U`` holding U^0 (updated in place). Start from centers: ``V0`` [C].
        ``U`` (allocated when None) receives U^k and ``V`` (allocated when
        None, or V0 itself) receives V^k. ``recompute=True`` keeps no U
        between iterations (``FCM_OPT_RECOMPUTE``). ``deterministic=True``
        deals every tile of the whole-run kernel in fixed warp shares, so
        large images give bit-identical results run after run
        (``FCM_OPT_DETERMINISTIC``).
        """
        import torch
        n = _numel(x)

        def alloc(shape):
            # outputs follow the kind of x: CUDA tensor, (pinned) CPU tensor or numpy
            if isinstance(x, torch.Tensor):
                t = torch.empty(shape, dtype=torch.float32, device=x.device)
                return t.pin_memory() if (not x.is_cuda and x.is_pinned()) else t
            return np.empty(shape, dtype=np.float32)

        if V0 is not None:
            mode = _lib.FCM_INIT_V
            if V is None:
                V = V0
            elif V is not V0:
                V[...] = V0
            u0p = None
        else:
            mode = _lib.FCM_INIT_U
            if U0 is None and U is None:
                raise ValueError("give U0, V0, or U holding U^0")
            u0p = U0
        if U is None:
            U = alloc((C, n))
        if V is None:
            V = alloc((C,))
        if _numel(U) != C * n or _numel(V) != C or (u0p is not None and _numel(u0p) != C * n):
            raise ValueError("U and U0 must hold C*n floats and V C floats")
        opts = ((_lib.FCM_OPT_TRACE if trace else 0) | (0 if graph else _lib.FCM_OPT_NO_GRAPH)
                | (0 if tma else _lib.FCM_OPT_NO_TMA) | (0 if persistent else _lib.FCM_OPT_NO_PERSISTENT)
                | (_lib.FCM_OPT_RECOMPUTE if recompute else 0)
                | (_lib.FCM_OPT_DETERMINISTIC if deterministic else 0))
        rep = _lib.fcm_report()
        self._bind_stream()
        st = self._lib.fcm_run(self._h, _ptr(x), n, int(C), float(m), float(eps), int(max_iter),
                               mode, None if u0p is None else _ptr(u0p), _ptr(U), _ptr(V), opts,
                               ctypes.byref(rep))
        if raise_on_error:
            _lib.check(st, self._h)
        tr = None
        if trace and st >= 0:
            k = rep.iters
            d = np.zeros(k)
            J = np.zeros(k)
            Vt = np.zeros((k, C))
            got = self._lib.fcm_get_trace(self._h, d.ctypes.data_as(_lib._dp),
                                          J.ctypes.data_as(_lib._dp), Vt.ctypes.data_as(_lib._dp), k)
            _lib.check(got, self._h)
            tr = {"delta": d[:got], "J": J[:got], "V": Vt[:got]}
        return FCMResult(U=U, V=V, iters=rep.iters, status=st, delta=rep.delta, J=rep.J,
                         V64=np.array(rep.V64[:C]), flags=rep.flags, launches=rep.launches, trace=tr)

    def init_dirichlet(self, n: int, C: int, seed: int, U=None):
        """The seeded random U^0 of Algorithm 1 step 2, drawn on the device
        (``fcm_init_dirichlet``) into ``U`` [C, n] (allocated when None)."""
        import torch
        if U is None:
            U = torch.empty((C, n), dtype=torch.float32, device=torch.device("cuda", self.device))
        if _numel(U) != C * n:
            raise ValueError("U must hold C*n floats")
        self._bind_stream()
        _lib.check(self._lib.fcm_init_dirichlet(self._h, int(n), int(C), int(seed), _ptr(U)), self._h)
        return U

    def run_seeded(self, x, C: int, m: float = 2.0, eps: float = 1e-5, max_iter: int = 300, *, seed: int,
                   U=None, V=None, raise_on_error: bool = True) -> FCMResult:
        """Algorithm 1 from the seeded random start drawn on the device
        (``fcm_run_seeded``); ``U`` receives U^k (allocated when None)."""
        import torch
        n = _numel(x)
        dev = torch.device("cuda", self.device)
        if U is None:
            U = torch.empty((C, n), dtype=torch.float32, device=dev)
        if V is None:
            V = torch.empty(C, dtype=torch.float32, device=dev)
        rep = _lib.fcm_report()
        self._bind_stream()
        st = self._lib.fcm_run_seeded(self._h, _ptr(x), n, int(C), float(m), float(eps), int(max_iter), int(seed),
                                      _ptr(U), _ptr(V), 0, ctypes.byref(rep))
        if raise_on_error:
            _lib.check(st, self._h)
        return FCMResult(U=U, V=V, iters=rep.iters, status=st, delta=rep.delta, J=rep.J,
                         V64=np.array(rep.V64[:C]), flags=rep.flags, launches=rep.launches, trace=None)

    def run_stream(self, xs, C: int, m: float = 2.0, eps: float = 1e-5, max_iter: int = 300, *,
                   U0s=None, Us=None, V=None, recompute: bool = False,
                   deterministic: bool = False, raise_on_error: bool = True) -> list[FCMResult]:
        """Algorithm 1 on a sequence of same-sized images in host memory
        (``fcm_run_stream``): the upload of the next image and the download
        of the previous one overlap the current run.

        ``xs``: list of n float32 pixels each (pinned CPU tensors copy
        fastest; numpy arrays work). ``U0s``: list of [C, n] initial
        memberships (read only), or None with each ``Us[i]`` holding U^0.
        ``Us`` (allocated like ``xs[0]`` when None) receives each U^k; ``V``
        ([len(xs), C], allocated when None) receives each V^k.
        """
        import torch
        k = len(xs)
        if k < 1:
            raise ValueError("give at least one image")
        n = _numel(xs[0])
        if any(_numel(x) != n for x in xs):
            raise ValueError("every image must hold the same number of pixels")

        def alloc(shape, like):
            if isinstance(like, torch.Tensor):
                t = torch.empty(shape, dtype=torch.float32)
                return t.pin_memory() if like.is_pinned() else t
            return np.empty(shape, dtype=np.float32)

        if U0s is None and Us is None:
            raise ValueError("give U0s, or Us holding U^0")
        if U0s is not None and (len(U0s) != k or any(_numel(u) != C * n for u in U0s)):
            raise ValueError("U0s must hold one [C, n] array per image")
        if Us is None:
            Us = [alloc((C, n), xs[0]) for _ in range(k)]
        if len(Us) != k or any(_numel(u) != C * n for u in Us):
            raise ValueError("Us must hold one [C, n] array per image")
        if V is None:
            V = np.empty((k, C), dtype=np.float32)
        if _numel(V) != k * C or (isinstance(V, torch.Tensor) and V.is_cuda):
            raise ValueError("V must be a host array of len(xs) x C floats")
        ptrs = lambda arrs: (_lib._vp * k)(*[_ptr(a) for a in arrs])
        xp, up = ptrs(xs), ptrs(Us)
        u0p = ptrs(U0s) if U0s is not None else None
        reps = (_lib.fcm_report * k)()
        self._bind_stream()
        st = self._lib.fcm_run_stream(self._h, k, xp, n, int(C), float(m), float(eps), int(max_iter),
                                      u0p, up, _ptr(V),
                                      (_lib.FCM_OPT_RECOMPUTE if recompute else 0)
                                      | (_lib.FCM_OPT_DETERMINISTIC if deterministic else 0), reps)
        if raise_on_error:
            _lib.check(st, self._h)
        return [FCMResult(U=Us[i], V=V[i], iters=reps[i].iters, status=reps[i].status, delta=reps[i].delta,
                          J=reps[i].J, V64=np.array(reps[i].V64[:C]), flags=reps[i].flags,
                          launches=reps[i].launches) for i in range(k)]

    def run_hist(self, x, C: int, m: float = 2.0, eps: float = 1e-5, max_iter: int = 300, *,
                 U0=None, V0=None, U=None, V=None, raise_on_error: bool = True) -> FCMResult:
        """Algorithm 1 on the 256-bin histogram (``fcm_run_hist``) for x that
        holds integer grey levels 0..255. Same arguments and result as
        ``run``; x, U and U0 must be CUDA tensors."""
        import torch
        n = _numel(x)
        if V0 is not None:
            mode = _lib.FCM_INIT_V
            if V is None:
                V = V0
            elif V is not V0:
                V[...] = V0
            u0p = None
        else:
            mode = _lib.FCM_INIT_U
            if U0 is None and U is None:
                raise ValueError("give U0, V0, or U holding U^0")
            u0p = U0
        if U is None:
            U = torch.empty((C, n), dtype=torch.float32, device=x.device)
        if V is None:
            V = torch.empty(C, dtype=torch.float32, device=x.device)
        if _numel(U) != C * n or _numel(V) != C or (u0p is not None and _numel(u0p) != C * n):
            raise ValueError("U and U0 must hold C*n floats and V C floats")
        rep = _lib.fcm_report()
        self._bind_stream()
        st = self._lib.fcm_run_hist(self._h, _ptr(x), n, int(C), float(m), float(eps), int(max_iter), mode,
                                    None if u0p is None else _ptr(u0p), _ptr(U), _ptr(V), ctypes.byref(rep))
        if raise_on_error:
            _lib.check(st, self._h)
        return FCMResult(U=U, V=V, iters=rep.iters, status=st, delta=rep.delta, J=rep.J,
                         V64=np.array(rep.V64[:C]), flags=rep.flags, launches=rep.launches, trace=None)

    def run_multi(self, x, C: int, m: float = 2.0, eps: float = 1e-5, max_iter: int = 300, *,
                  U0=None, V0=None, U=None, V=None, raise_on_error: bool = True) -> FCMResult:
        """Algorithm 1 on pixels of D channels (``fcm_run_multi``): ``x`` is a
        CUDA tensor [D, n]; ``V0``/``V`` are [C, D]; ``U0``/``U`` [C, n]. The
        result's V64 holds the FP64 centers, shape [C, D]."""
        import torch
        D, n = int(x.shape[0]), int(x.shape[1])
        if V0 is not None:
            mode = _lib.FCM_INIT_V
            if V is None:
                V = V0
            elif V is not V0:
                V[...] = V0
            u0p = None
        else:
            mode = _lib.FCM_INIT_U
            if U0 is None and U is None:
                raise ValueError("give U0, V0, or U holding U^0")
            u0p = U0
        if U is None:
            U = torch.empty((C, n), dtype=torch.float32, device=x.device)
        if V is None:
            V = torch.empty((C, D), dtype=torch.float32, device=x.device)
        if _numel(U) != C * n or _numel(V) != C * D or (u0p is not None and _numel(u0p) != C * n):
            raise ValueError("U and U0 must hold C*n floats and V C*D floats")
        v64 = np.empty(C * D)
        rep = _lib.fcm_report()
        self._bind_stream()
        st = self._lib.fcm_run_multi(self._h, _ptr(x), n, D, int(C), float(m), float(eps), int(max_iter), mode,
                                     None if u0p is None else _ptr(u0p), _ptr(U), _ptr(V),
                                     v64.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(rep))
        if raise_on_error:
            _lib.check(st, self._h)
        return FCMResult(U=U, V=V, iters=rep.iters, status=st, delta=rep.delta, J=rep.J,
                         V64=v64.reshape(C, D), flags=rep.flags, launches=rep.launches, trace=None)

    def dsc(self, U, truth, n_classes: int, class_of_cluster=None, V=None):
        """Dice similarity per class of the defuzzified U against ``truth``
        (``fcm_dsc``). ``class_of_cluster`` maps clusters to classes; when it
        is None, clusters are matched to classes by ascending center (``V``),
        for classes numbered in ascending order of intensity. Returns
        (dsc [n_classes], counts [n_classes, 3] of |PR|, |GT|, |PR n GT|)."""
        C = int(U.shape[0])
        n = _numel(U) // C
        if class_of_cluster is None:
            order = np.argsort(np.asarray(V.cpu() if hasattr(V, "cpu") else V, dtype=np.float64).reshape(-1))
            class_of_cluster = np.empty(C, dtype=np.int32)
            class_of_cluster[order] = np.arange(C)
        cmap = np.ascontiguousarray(class_of_cluster, dtype=np.int32)
        out = np.empty(n_classes)
        counts = np.empty(3 * n_classes, dtype=np.int64)
        self._bind_stream()
        _lib.check(self._lib.fcm_dsc(self._h, _ptr(U), n, C, ctypes.c_void_p(truth.data_ptr()),
                                     cmap.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(n_classes),
                                     counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self._h)
        return out, counts.reshape(n_classes, 3)

    def time_pass(self, x, C: int, m: float, U, V, launches: int = 20, tma: bool = True) -> float:
        """Average milliseconds per launch of the iteration pass, from
        ``launches`` back-to-back launches timed with CUDA events (U updated in
        place, no stopping test). A profiling aid."""
        ms = ctypes.c_float(0.0)
        self._bind_stream()
        _lib.check(self._lib.fcm_time_pass(self._h, _ptr(x), _numel(x), int(C), float(m), _ptr(U),
                                           _ptr(V), int(launches), 0 if tma else _lib.FCM_OPT_NO_TMA,
                                           ctypes.byref(ms)), self._h)
        return ms.value

    @staticmethod
    def _c_slices(slices):
        """The fcm_slice array of a batch, as a numpy structured array (its
        memory is what the library reads and writes)."""
        import torch
        for s in slices:
            if s.U is None:
                s.U = torch.empty((s.C, _numel(s.x)), dtype=torch.float32, device=s.x.device)
            if s.V is None:
                s.V = torch.empty(s.C, dtype=torch.float32, device=s.x.device)
        a = np.zeros(len(slices), dtype=_SLICE_DTYPE)
        a["x"] = [_ptr(s.x) for s in slices]
        a["n"] = [_numel(s.x) for s in slices]
        a["C"] = [s.C for s in slices]
        a["m"] = [s.m for s in slices]
        a["eps"] = [s.eps for s in slices]
        a["max_iter"] = [s.max_iter for s in slices]
        a["U"] = [_ptr(s.U) for s in slices]
        a["V"] = [_ptr(s.V) for s in slices]
        a["U0"] = [0 if s.U0 is None else _ptr(s.U0) for s in slices]
        a["init_mode"] = [_lib.FCM_INIT_U if s.V0 is None else _lib.FCM_INIT_V for s in slices]
        for i, s in enumerate(slices):
            if s.V0 is not None:
                v0 = np.asarray(s.V0, dtype=np.float64).reshape(-1)[:s.C]
                a["V0"][i, :v0.size] = v0
        return a

    @staticmethod
    def _arr_ptr(a):
        return a.ctypes.data_as(ctypes.POINTER(_lib.fcm_slice))

    @staticmethod
    def _read_back(a, slices):
        iters, status, flags = a["iters"].tolist(), a["status"].tolist(), a["flags"].tolist()
        delta, J, modes = a["delta"].tolist(), a["J"].tolist(), a["init_mode"].tolist()
        V64, V0 = a["V64"].copy(), a["V0"]
        for i, s in enumerate(slices):
            s.iters, s.status, s.flags, s.delta, s.J = iters[i], status[i], flags[i], delta[i], J[i]
            s.V64 = V64[i, :s.C]
            warm = modes[i] == _lib.FCM_INIT_V and s.V0 is None
            s.init = "V" if modes[i] == _lib.FCM_INIT_V else "U"
            s.V0_warm = V0[i, :s.C].copy() if warm else None

    def _batch_opts(self, tune, retune, graph, presolve=False):
        return ((0 if tune else _lib.FCM_BATCH_NO_TUNE) | (_lib.FCM_BATCH_RETUNE if retune else 0)
                | (0 if graph else _lib.FCM_BATCH_NO_GRAPH) | (_lib.FCM_BATCH_PRESOLVE if presolve else 0))

    def run_batched(self, slices, tune: bool = True, retune: bool = False, graph: bool = True,
                    raise_on_error: bool = False, read_back: bool = True, presolve: bool = False) -> int:
        """Algorithm 1 on every slice in one persistent launch (see
        ``fcm_run_batched``). Fills each Slice's U, V and result fields and
        returns the aggregate status. With a ``Batch`` and ``read_back=False``
        the per-slice results stay in ``batch.arr`` (host memory) until
        ``batch.read_back()``; U and V are written either way."""
        b = _as_batch(slices)
        self._bind_stream()
        st = self._lib.fcm_run_batched(self._h, self._arr_ptr(b.arr), len(b),
                                       self._batch_opts(tune, retune, graph, presolve))
        if st in (_lib.FCM_ERR_INVALID_ARG, _lib.FCM_ERR_CUDA, _lib.FCM_ERR_OOM) or raise_on_error:
            _lib.check(st, self._h)
        if read_back or not isinstance(slices, Batch):
            b.read_back()
        return st

    def run_batched_hist(self, slices, raise_on_error: bool = False, read_back: bool = True) -> int:
        """Algorithm 1 on the 256-bin histogram of every slice of a batch of
        8-bit slices, one CTA per slice (see ``fcm_run_batched_hist``). Same
        slices, fields and return value as ``run_batched``."""
        b = _as_batch(slices)
        self._bind_stream()
        st = self._lib.fcm_run_batched_hist(self._h, self._arr_ptr(b.arr), len(b))
        if st in (_lib.FCM_ERR_INVALID_ARG, _lib.FCM_ERR_CUDA, _lib.FCM_ERR_OOM) or raise_on_error:
            _lib.check(st, self._h)
        if read_back or not isinstance(slices, Batch):
            b.read_back()
        return st

    def run_batched_warm(self, slices, tune: bool = True, retune: bool = False, graph: bool = True,
                         read_back: bool = True):
        """Warm-started batch (``fcm_run_batched_warm``): predicted V^0, with the
        plain cold start (each slice's U0) as the fallback. Returns
        (status, number of slices that ran cold). ``s.init`` tells which."""
        b = _as_batch(slices)
        cold = ctypes.c_int(0)
        self._bind_stream()
        st = self._lib.fcm_run_batched_warm(self._h, self._arr_ptr(b.arr), len(b),
                                            self._batch_opts(tune, retune, graph), ctypes.byref(cold))
        if st in (_lib.FCM_ERR_INVALID_ARG, _lib.FCM_ERR_CUDA, _lib.FCM_ERR_OOM):
            _lib.check(st, self._h)
        if read_back or not isinstance(slices, Batch):
            b.read_back()
        return st, cold.value

    # ---- warm-start network ------------------------------------------------

    def model_init(self, seed: int = 0):
        _lib.check(self._lib.fcm_model_init(self._h, int(seed)), self._h)

    def model_params(self) -> np.ndarray:
        p = np.empty(_lib.FCM_MODEL_PARAMS, dtype=np.float32)
        _lib.check(self._lib.fcm_model_get_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                  p.size), self._h)
        return p

    def set_model_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        _lib.check(self._lib.fcm_model_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                  p.size), self._h)

    def model_save(self, path: str):
        _lib.check(self._lib.fcm_model_save(self._h, str(path).encode()), self._h)

    def model_load(self, path: str):
        _lib.check(self._lib.fcm_model_load(self._h, str(path).encode()), self._h)

    def features(self, slices):
        """Network inputs [n, 264] (CUDA tensor) of the slices' x and C."""
        import torch
        arr = self._c_slices(slices)
        out = torch.empty((len(slices), _lib.MODEL_D_IN), dtype=torch.float32, device=slices[0].x.device)
        self._bind_stream()
        _lib.check(self._lib.fcm_features(self._h, self._arr_ptr(arr), len(slices), _ptr(out)), self._h)
        return out

    def model_forward(self, feats):
        import torch
        out = torch.empty((feats.shape[0], _lib.MODEL_D_OUT), dtype=torch.float32, device=feats.device)
        self._bind_stream()
        _lib.check(self._lib.fcm_model_forward(self._h, _ptr(feats), feats.shape[0], _ptr(out)), self._h)
        return out

    def model_loss_grad(self, feats, targets, Cs):
        g = np.empty(_lib.FCM_MODEL_PARAMS, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        self._bind_stream()
        _lib.check(self._lib.fcm_model_loss_grad(
            self._h, _ptr(feats), _ptr(targets), ctypes.c_void_p(Cs.data_ptr()), feats.shape[0],
            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)), self._h)
        return loss.value, g

    def model_train(self, feats, targets, Cs, epochs: int, batch: int = 256, lr: float = 1e-3,
                    seed: int = 0) -> float:
        loss = ctypes.c_float(0.0)
        self._bind_stream()
        _lib.check(self._lib.fcm_model_train(self._h, _ptr(feats), _ptr(targets), ctypes.c_void_p(Cs.data_ptr()),
                                             feats.shape[0], int(epochs), int(batch), float(lr), int(seed),
                                             ctypes.byref(loss)), self._h)
        return loss.value

    def predict_centers(self, slices):
        """Sets each slice's V0 to the network's prediction."""
        arr = self._c_slices(slices)
        self._bind_stream()
        _lib.check(self._lib.fcm_predict_centers(self._h, self._arr_ptr(arr), len(slices)), self._h)
        for i, s in enumerate(slices):
            s.V0 = arr["V0"][i, :s.C].copy()

    def batched_plan(self) -> dict:
        p = _lib.fcm_batch_plan()
        _lib.check(self._lib.fcm_batched_plan(self._h, ctypes.byref(p)), self._h)
        names = {_lib.FCM_SCHED_SLICES: "slices", _lib.FCM_SCHED_ROUNDS: "rounds", _lib.FCM_SCHED_TEAMS: "teams"}
        return {"schedule": names[p.schedule],
                "block": p.block, "cluster": p.cluster, "big": p.big, "tile": p.tile, "ms": p.ms}

    def set_batched_plan(self, block=None, cluster=1, big=1 << 62, schedule="slices", tile=0):
        """Force a launch shape for later batched runs; no arguments returns
        to the autotuner. ``schedule="rounds"`` takes ``block`` and ``tile``;
        ``"teams"`` takes ``block`` and ``tile`` (the team-size target in
        percent of the mean cost per CTA); ``"slices"`` takes ``block``,
        ``cluster``, ``big`` and ``tile`` (0, or the first-phase iteration cap
        of a two-phase batch)."""
        if block is None:
            _lib.check(self._lib.fcm_batched_set_plan(self._h, None), self._h)
            return
        codes = {"slices": _lib.FCM_SCHED_SLICES, "rounds": _lib.FCM_SCHED_ROUNDS, "teams": _lib.FCM_SCHED_TEAMS}
        sliced = schedule == "slices"
        p = _lib.fcm_batch_plan(int(block), int(cluster) if sliced else 1, int(big) if sliced else 0, 0.0,
                                codes[schedule], int(tile))
        _lib.check(self._lib.fcm_batched_set_plan(self._h, ctypes.byref(p)), self._h)
