"""Thin ctypes binding of libfresnel (include/fresnel.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libfresnel.so.  PyTorch supplies device memory and the CUDA stream.
If the library is missing this module raises; there is no CPU fallback.

Names follow the C ABI: ``fresnel_plan``, ``fresnel_plan_many``,
``fresnel_eval``, ``fresnel_eval_many``, ``fresnel_eval_host``,
``fresnel_check``, ``fresnel_destroy``, ``fresnel_last_error``,
``fresnel_get_info``, ``fresnel_get_nodes``; the ``Plan`` and ``BatchPlan``
classes wrap them for convenience.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfresnel.so")

FRESNEL_OK = 0
STATUS_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_TIMEOUT",
                -5: "ERR_UNSUPPORTED", -6: "ERR_DEVICE"}
FAMILY_KINDS = {"fourier": 0, "line_rule": 1, "nodes": 2, "petals": 3, "triangles": 4}
PRECISIONS = {"fp64": 0, "fp32": 1}
OUTPUTS = {"aperture": 0, "occulter": 1}
GRID, SCATTERED = 0, 1


class FresnelError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Family(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_panels", ctypes.c_int), ("p", ctypes.c_int),
                ("m", ctypes.c_int), ("params", ctypes.POINTER(ctypes.c_double)),
                ("n_params", ctypes.c_longlong), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("motion", ctypes.POINTER(ctypes.c_double))]


class Problem(ctypes.Structure):
    _fields_ = [("families", ctypes.POINTER(Family)), ("n_families", ctypes.c_int),
                ("lam", ctypes.c_double), ("z", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("output", ctypes.c_int),
                ("target_kind", ctypes.c_int), ("grid_n1", ctypes.c_int),
                ("grid_n2", ctypes.c_int), ("grid_h", ctypes.c_double),
                ("grid_x0", ctypes.c_double), ("grid_y0", ctypes.c_double),
                ("box", ctypes.c_double * 4), ("sigma", ctypes.c_double),
                ("kernel_w", ctypes.c_int), ("recompute_nodes", ctypes.c_int),
                ("sync_status", ctypes.c_int), ("max_device_bytes", ctypes.c_longlong),
                ("t3_binning", ctypes.c_int), ("fft_split_above", ctypes.c_int),
                ("autotune", ctypes.c_int), ("nsli_far", ctypes.c_double),
                ("screen_amp", ctypes.c_void_p), ("screen_opd", ctypes.c_void_p),
                ("screen_n1", ctypes.c_int), ("screen_n2", ctypes.c_int),
                ("screen_box", ctypes.c_double * 4), ("max_spin", ctypes.c_longlong),
                ("deterministic", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_longlong), ("w", ctypes.c_int), ("beta", ctypes.c_double),
                ("sigma", ctypes.c_double), ("nf1", ctypes.c_int), ("nf2", ctypes.c_int),
                ("nfft1", ctypes.c_int), ("nfft2", ctypes.c_int), ("tile_x", ctypes.c_int),
                ("tile_y", ctypes.c_int), ("device_bytes", ctypes.c_longlong),
                ("launches_per_eval", ctypes.c_int), ("split_tiles", ctypes.c_int),
                ("max_tile_records", ctypes.c_int), ("t3_binning", ctypes.c_int),
                ("live_tile_rows", ctypes.c_int)]


EXPORTS = ["fresnel_default_opts", "fresnel_plan", "fresnel_plan_many", "fresnel_eval",
           "fresnel_eval_many", "fresnel_eval_many_scattered", "fresnel_eval_host",
           "fresnel_grad_profile", "fresnel_grad_shape", "fresnel_nsli",
           "fresnel_check", "fresnel_destroy", "fresnel_last_error", "fresnel_get_info",
           "fresnel_get_nodes", "fresnel_set_timing", "fresnel_stage_times", "fresnel_spread",
           "fresnel_spread_noalloc"]

_lib = None


def load_library(path=LIB_PATH):
    """Load libfresnel.so (built in-tree by paper_2010_05978_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FresnelError(-2, "libfresnel.so not found at %s; build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    vp, ll, d = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double
    lib.fresnel_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.fresnel_default_opts.restype = None
    lib.fresnel_plan.argtypes = [ctypes.POINTER(Family), ctypes.c_int, d, d, d,
                                 ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    lib.fresnel_plan.restype = ctypes.c_int
    lib.fresnel_plan_many.argtypes = [ctypes.POINTER(Problem), ctypes.c_int, d,
                                      ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    lib.fresnel_plan_many.restype = ctypes.c_int
    lib.fresnel_eval.argtypes = [vp, vp, ll, vp]
    lib.fresnel_eval.restype = ctypes.c_int
    lib.fresnel_eval_many.argtypes = [vp, vp]
    lib.fresnel_eval_many.restype = ctypes.c_int
    lib.fresnel_eval_many_scattered.argtypes = [vp, vp, ctypes.POINTER(ll), vp]
    lib.fresnel_eval_many_scattered.restype = ctypes.c_int
    lib.fresnel_grad_profile.argtypes = [vp, vp, vp]
    lib.fresnel_grad_profile.restype = ctypes.c_int
    lib.fresnel_grad_shape.argtypes = [vp, vp, vp]
    lib.fresnel_grad_shape.restype = ctypes.c_int
    lib.fresnel_nsli.argtypes = [vp, vp, ll, vp]
    lib.fresnel_nsli.restype = ctypes.c_int
    lib.fresnel_eval_host.argtypes = [vp, vp, ll, vp]
    lib.fresnel_eval_host.restype = ctypes.c_int
    lib.fresnel_check.argtypes = [vp]
    lib.fresnel_check.restype = ctypes.c_int
    lib.fresnel_destroy.argtypes = [vp]
    lib.fresnel_destroy.restype = ctypes.c_int
    lib.fresnel_last_error.argtypes = []
    lib.fresnel_last_error.restype = ctypes.c_char_p
    lib.fresnel_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    lib.fresnel_get_info.restype = ctypes.c_int
    lib.fresnel_get_nodes.argtypes = [vp, vp, vp, vp]
    lib.fresnel_get_nodes.restype = ctypes.c_int
    lib.fresnel_set_timing.argtypes = [vp, ctypes.c_int]
    lib.fresnel_set_timing.restype = ctypes.c_int
    lib.fresnel_stage_times.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_char_p),
                                        ctypes.c_int]
    lib.fresnel_stage_times.restype = ctypes.c_int
    lib.fresnel_spread.argtypes = [vp, vp, vp, ll, ctypes.c_int, ctypes.c_int, ctypes.c_int, d,
                                   vp, vp]
    lib.fresnel_spread.restype = ctypes.c_int
    lib.fresnel_spread_noalloc.argtypes = lib.fresnel_spread.argtypes
    lib.fresnel_spread_noalloc.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status):
    if status != FRESNEL_OK:
        raise FresnelError(status, load_library().fresnel_last_error().decode())


def family_params(fam):
    """(kind, n_panels, p, m, params, cx, cy) of a panel-family dict."""
    kind = fam["kind"]
    if kind == "fourier":
        params = np.ascontiguousarray(fam["params"], dtype=np.float64)
        return 0, fam["n_panels"], fam["p"], fam["m"], params, fam.get("cx", 0.0), fam.get("cy", 0.0)
    if kind == "line_rule":
        params = np.ascontiguousarray(np.concatenate(
            [np.asarray(fam[k], np.float64) for k in ("X", "Y", "W", "V")]))
        n = len(fam["X"])
        return 1, n, 1, fam["m"], params, fam.get("cx", 0.0), fam.get("cy", 0.0)
    if kind == "nodes":
        params = np.ascontiguousarray(np.concatenate(
            [np.asarray(fam[k], np.float64) for k in ("x", "y", "w")]))
        return 2, 0, 0, 0, params, 0.0, 0.0
    if kind == "triangles":
        tri = np.ascontiguousarray(np.asarray(fam["tri"], np.float64).reshape(-1, 6).ravel())
        return 4, len(tri) // 6, fam["p"], 0, tri, fam.get("cx", 0.0), fam.get("cy", 0.0)
    if kind == "petals":
        prof = fam["profile"]
        if prof["kind"] == "hg":
            code, data = 0, [prof["b"], prof["q"]]
        elif prof["kind"] == "bspline":
            code, data = 1, prof["coefs"]
        elif prof["kind"] == "table":
            code, data = 2, prof["A"]
        else:
            raise ValueError("unknown petal profile %r" % prof["kind"])
        head = [fam["a"], fam["R"], fam.get("n_d", 0), fam.get("m_d", 0), code]
        params = np.ascontiguousarray(np.concatenate(
            [np.asarray(head, np.float64), np.asarray(data, np.float64)]))
        return 3, fam["n_petals"], fam["n_p"], fam["m"], params, fam.get("cx", 0.0), fam.get("cy", 0.0)
    raise ValueError("unknown family kind %r" % kind)


def _family_array(families):
    """ctypes array of Family structs and the numpy params it points into."""
    fams = (Family * len(families))()
    keep = []
    for i, f in enumerate(families):
        kind, npan, p, m, params, cx, cy = family_params(f)
        keep.append(params)
        motion = None
        if f.get("motion") is not None:   # petals: (n_petals, 3) rows phi, tx, ty
            mo = np.ascontiguousarray(np.asarray(f["motion"], np.float64).ravel())
            keep.append(mo)
            motion = mo.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        fams[i] = Family(kind, int(npan), int(p), int(m),
                         params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         len(params), float(cx), float(cy), motion)
    return fams, keep


def _make_opts(lib, precision, output, grid, box, sigma, kernel_w, recompute_nodes, sync_status,
               max_device_bytes, t3_binning, fft_split_above=0, autotune=False, nsli_far=0.0,
               screen=None, max_spin=0, deterministic=False):
    o = Opts()
    lib.fresnel_default_opts(ctypes.byref(o))
    o.precision = PRECISIONS[precision]
    o.output = OUTPUTS[output]
    if grid is not None:
        o.target_kind = GRID
        o.grid_n1, o.grid_n2 = int(grid["n1"]), int(grid["n2"])
        o.grid_h = float(grid["h"])
        o.grid_x0, o.grid_y0 = float(grid.get("x0", 0.0)), float(grid.get("y0", 0.0))
    else:
        o.target_kind = SCATTERED
        for i in range(4):
            o.box[i] = float(box[i])
    o.sigma = float(sigma)
    o.kernel_w = int(kernel_w)
    o.recompute_nodes = int(bool(recompute_nodes))
    o.sync_status = int(bool(sync_status))
    o.max_device_bytes = int(max_device_bytes)
    o.t3_binning = int(t3_binning)
    o.fft_split_above = int(fft_split_above)
    o.autotune = int(bool(autotune))
    o.nsli_far = float(nsli_far)
    o.max_spin = int(max_spin)
    o.deterministic = int(bool(deterministic))
    o._keep = []
    if screen is not None:
        # dict(amp=, opd=, box=(x0, x1, y0, y1)): 2D arrays (n2 rows of n1)
        arrs = {k: np.ascontiguousarray(screen[k], dtype=np.float64)
                for k in ("amp", "opd") if screen.get(k) is not None}
        if not arrs:
            raise ValueError("screen needs amp and/or opd")
        shp = next(iter(arrs.values())).shape
        if len(shp) != 2 or any(a.shape != shp for a in arrs.values()):
            raise ValueError("screen arrays must be 2D and of one shape")
        o.screen_n2, o.screen_n1 = int(shp[0]), int(shp[1])
        o.screen_amp = arrs["amp"].ctypes.data if "amp" in arrs else None
        o.screen_opd = arrs["opd"].ctypes.data if "opd" in arrs else None
        for i in range(4):
            o.screen_box[i] = float(screen["box"][i])
        o._keep = list(arrs.values())
    return o


def _profile_sizes(families):
    """Profile data length of each PETALS family (the gradient layout)."""
    return [len(family_params(f)[4]) - 5 for f in families if f["kind"] == "petals"]


def _shape_sizes(families):
    """Coefficient count of each FOURIER family (the shape-gradient layout)."""
    return [len(family_params(f)[4]) for f in families if f["kind"] == "fourier"]


class _PlanHandle:
    """Methods shared by single and batched plans."""

    def grad_profile(self, gamma):
        """dL/d(profile data) of every PETALS family (FP64 CUDA tensor, families
        concatenated in plan order) for dL = Re sum conj(gamma) du, gamma shaped
        like the output (torch's gradient convention for complex tensors)."""
        torch = self._torch
        gamma = gamma.to(self.cdtype).contiguous()
        out = torch.empty(max(1, sum(self.profile_sizes)), dtype=torch.float64, device="cuda")
        _check(load_library().fresnel_grad_profile(self.handle, gamma.data_ptr(), out.data_ptr()))
        return out[:sum(self.profile_sizes)]

    def grad_shape(self, gamma):
        """dL/d(boundary coefficients) of every FOURIER family (FP64 CUDA tensor,
        each family's [r0, a1, b1, ...] concatenated in plan order) for
        dL = Re sum conj(gamma) du, gamma shaped like the output."""
        torch = self._torch
        gamma = gamma.to(self.cdtype).contiguous()
        out = torch.empty(max(1, sum(self.shape_sizes)), dtype=torch.float64, device="cuda")
        _check(load_library().fresnel_grad_shape(self.handle, gamma.data_ptr(), out.data_ptr()))
        return out[:sum(self.shape_sizes)]

    def check(self):
        _check(load_library().fresnel_check(self.handle))

    def info(self):
        inf = Info()
        _check(load_library().fresnel_get_info(self.handle, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    def nodes(self):
        """The plan's quadrature nodes (x, y, w) as float64 CUDA tensors."""
        torch = self._torch
        n = self.info()["n_nodes"]
        x, y, w = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
        _check(load_library().fresnel_get_nodes(self.handle, x.data_ptr(), y.data_ptr(),
                                                w.data_ptr()))
        return x, y, w

    def set_timing(self, enable=True):
        load_library().fresnel_set_timing(self.handle, int(enable))

    def stage_times(self):
        ms = (ctypes.c_double * 16)()
        names = (ctypes.c_char_p * 16)()
        n = load_library().fresnel_stage_times(self.handle, ms, names, 16)
        return {names[i].decode(): ms[i] for i in range(n)}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load_library().fresnel_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan(_PlanHandle):
    """Several independent problems in one plan (``fresnel_plan_many``).

    problems: list of dicts {"families": [...], "lam": lambda, "z": z}; the
    other arguments as for ``Plan``.  With grid=...: ``eval()`` returns a
    CUDA tensor of shape (n_problems, n2, n1).  With box=...: ``eval(targets,
    counts)`` takes every problem's targets concatenated (float64 CUDA tensor
    (sum(counts), 2)) and returns the concatenated fields.
    """

    def __init__(self, problems, tol, precision="fp32", output="aperture", grid=None, box=None,
                 sigma=0.0, kernel_w=0, recompute_nodes=False, sync_status=True,
                 max_device_bytes=0, t3_binning=0, fft_split_above=0, autotune=False,
                 stream=None, nsli_far=0.0, screen=None, max_spin=0,
                 deterministic=False):
        import torch
        lib = load_library()
        self._torch = torch
        probs = (Problem * len(problems))()
        self.profile_sizes = [n for q in problems for n in _profile_sizes(q["families"])]
        self.shape_sizes = [n for q in problems for n in _shape_sizes(q["families"])]
        self._keep = []
        for b, q in enumerate(problems):
            fams, keep = _family_array(q["families"])
            self._keep.append((fams, keep))
            probs[b] = Problem(fams, len(q["families"]), float(q["lam"]), float(q["z"]))
        o = _make_opts(lib, precision, output, grid, box, sigma, kernel_w, recompute_nodes,
                       sync_status, max_device_bytes, t3_binning, fft_split_above, autotune,
                       nsli_far, screen, max_spin, deterministic)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.fresnel_plan_many(probs, len(problems), float(tol), ctypes.byref(o),
                                     ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)))
        self.handle = h
        self.precision = precision
        self.grid = grid
        self.n_problems = len(problems)
        self.cdtype = torch.complex64 if precision == "fp32" else torch.complex128

    def eval(self, targets=None, counts=None, out=None):
        torch = self._torch
        if self.grid is not None:
            shape = (self.n_problems, self.grid["n2"], self.grid["n1"])
            if out is None:
                out = torch.empty(shape, dtype=self.cdtype, device="cuda")
            assert out.is_cuda and out.is_contiguous() and tuple(out.shape) == shape
            _check(load_library().fresnel_eval_many(self.handle, out.data_ptr()))
            return out
        counts = [int(m) for m in counts]
        assert len(counts) == self.n_problems
        total = sum(counts)
        assert targets.dtype == torch.float64 and targets.is_cuda and targets.is_contiguous()
        assert tuple(targets.shape) == (total, 2)
        if out is None:
            out = torch.empty((total,), dtype=self.cdtype, device="cuda")
        M = (ctypes.c_longlong * self.n_problems)(*counts)
        _check(load_library().fresnel_eval_many_scattered(
            self.handle, targets.data_ptr() if total else None, M,
            out.data_ptr() if total else None))
        return out


class Plan(_PlanHandle):
    """A libfresnel plan on the current CUDA device and stream.

    families: list of panel-family dicts (see workloads.py); lam, z: wavelength
    and distance (only lam*z matters, eq. fres); tol: requested relative error;
    precision "fp32" (fast mode) or "fp64"; output "aperture" or "occulter";
    grid=dict(n1, n2, h, x0, y0) for type-1 targets, or box=(xmin, xmax,
    ymin, ymax) for scattered (type-3) targets.

    Family dicts: {"kind": "fourier", "params", "n_panels", "p", "m"},
    {"kind": "line_rule", "X", "Y", "W", "V", "m"}, {"kind": "nodes", "x",
    "y", "w"}, {"kind": "triangles", "tri" (T x 6 vertex coordinates), "p"},
    {"kind": "petals", "n_petals", "a", "R", "profile", "m", "n_p", "n_d",
    "m_d"}; all but nodes take a centre "cx", "cy", and petals an optional
    "motion" (n_petals x 3 rows phi, tx, ty: each petal rotated by phi about
    the centre and translated, with root-arc patches added, Sec. 5.1).

    Options: recompute_nodes regenerates nodes, chirps and bins at every
    evaluation; sync_status=False makes evaluations asynchronous (read the
    device status with check()); sigma, kernel_w override the NUFFT's
    upsampling and kernel width; t3_binning (-1 off, 0 auto, 1 on) buckets
    scattered targets; autotune measures candidate settings at plan time;
    nsli_far is the distance beyond which nsli() uses the shadow fix (eq. li
    with the rounded winding number); screen=dict(amp=, opd=, box=(x0, x1,
    y0, y1)) multiplies each node's weight by A e^{2 pi i OPD / lam} from
    sampled amplitude and optical path difference (n2 rows of n1 samples);
    max_spin bounds the spreading stage's one device-side wait (polls before
    FRESNEL_ERR_TIMEOUT; 0 the built-in ~1 s, < 0 none: tests of that path);
    deterministic=True makes the outputs repeat bit for bit (exact
    fixed-point sums in the spreading stage).
    """

    def __init__(self, families, lam, z, tol, precision="fp32", output="aperture", grid=None,
                 box=None, sigma=0.0, kernel_w=0, recompute_nodes=False, sync_status=True,
                 max_device_bytes=0, t3_binning=0, fft_split_above=0, autotune=False,
                 stream=None, nsli_far=0.0, screen=None, max_spin=0,
                 deterministic=False):
        import torch
        lib = load_library()
        self._torch = torch
        fams, keep = _family_array(families)
        self.profile_sizes = _profile_sizes(families)
        self.shape_sizes = _shape_sizes(families)
        o = _make_opts(lib, precision, output, grid, box, sigma, kernel_w, recompute_nodes,
                       sync_status, max_device_bytes, t3_binning, fft_split_above, autotune,
                       nsli_far, screen, max_spin, deterministic)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.fresnel_plan(fams, len(families), float(lam), float(z), float(tol),
                                ctypes.byref(o), ctypes.c_void_p(stream.cuda_stream),
                                ctypes.byref(h)))
        self.handle = h
        self.precision = precision
        self.grid = grid
        self.cdtype = torch.complex64 if precision == "fp32" else torch.complex128

    # -------------------------------------------------------------- evaluation
    def eval(self, targets=None, out=None):
        """u at the plan's targets as a CUDA tensor (complex64 / complex128).

        Grid plans return shape (n2, n1) (k1 fastest); scattered plans take a
        contiguous float64 CUDA tensor of shape (M, 2) and return shape (M,).
        """
        torch = self._torch
        if self.grid is not None:
            M = self.grid["n1"] * self.grid["n2"]
            shape = (self.grid["n2"], self.grid["n1"])
            tptr = None
        else:
            assert targets.dtype == torch.float64 and targets.is_cuda and targets.is_contiguous()
            assert targets.dim() == 2 and targets.shape[1] == 2
            M = targets.shape[0]
            shape = (M,)
            tptr = targets.data_ptr() if M > 0 else None
        if out is None:
            out = torch.empty(shape, dtype=self.cdtype, device="cuda")
        _check(load_library().fresnel_eval(self.handle, tptr, M, out.data_ptr() if M > 0 else None))
        return out

    def nsli(self, targets):
        """u at scattered targets by the line integral of eq. nsli (FP64,
        complex128 CUDA tensor), from the plan's boundary rules."""
        torch = self._torch
        assert targets.dtype == torch.float64 and targets.is_cuda and targets.is_contiguous()
        M = targets.shape[0]
        out = torch.empty((M,), dtype=torch.complex128, device="cuda")
        _check(load_library().fresnel_nsli(self.handle, targets.data_ptr() if M else None, M,
                                           out.data_ptr() if M else None))
        return out

    def eval_host(self, targets=None, out=None):
        """Same evaluation from HOST numpy arrays (copies inside the call).
        With sync_status=False the call returns once the work is queued: out
        is complete after the plan's stream is synchronised (pinned arrays,
        e.g. numpy views of pin_memory tensors, give asynchronous copies)."""
        npc = np.complex64 if self.precision == "fp32" else np.complex128
        if self.grid is not None:
            M = self.grid["n1"] * self.grid["n2"]
            shape = (self.grid["n2"], self.grid["n1"])
            tptr = None
        else:
            targets = np.ascontiguousarray(targets, dtype=np.float64)
            M = targets.shape[0]
            shape = (M,)
            tptr = targets.ctypes.data if M > 0 else None
        if out is None:
            out = np.empty(shape, dtype=npc)
        _check(load_library().fresnel_eval_host(self.handle, tptr, M,
                                                out.ctypes.data if M > 0 else None))
        return out


def profile_field(theta, make_plan):
    """The field of a starshade design as a differentiable function of its
    petal profile data theta (a float64 torch tensor).

    make_plan(theta_numpy) returns a Plan or BatchPlan (grid targets) whose
    PETALS families all take their profile data (e.g. B-spline coefficients)
    from theta.  Returns the output tensor; backward gives dL/dtheta through
    fresnel_grad_profile (summed over the families sharing theta)."""
    import torch

    class _ProfileField(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            plan = make_plan(th.detach().cpu().numpy().astype(np.float64))
            u = plan.eval()
            ctx.plan = plan
            return u

        @staticmethod
        def backward(ctx, grad_u):
            plan = ctx.plan
            g = plan.grad_profile(grad_u)
            n = theta.numel()
            assert all(k == n for k in plan.profile_sizes)
            gt = g.view(len(plan.profile_sizes), n).sum(0)
            return gt.to(theta.device, theta.dtype).view_as(theta)

    return _ProfileField.apply(theta)


def shape_field(theta, make_plan):
    """The field of an aperture as a differentiable function of its Fourier
    boundary coefficients theta = [r0, a1, b1, ...] (a float64 torch tensor).

    make_plan(theta_numpy) returns a Plan or BatchPlan (grid targets) whose
    FOURIER families all take their params from theta.  Returns the output
    tensor; backward gives dL/dtheta through fresnel_grad_shape (summed over
    the families sharing theta)."""
    import torch

    class _ShapeField(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            plan = make_plan(th.detach().cpu().numpy().astype(np.float64))
            u = plan.eval()
            ctx.plan = plan
            return u

        @staticmethod
        def backward(ctx, grad_u):
            plan = ctx.plan
            g = plan.grad_shape(grad_u)
            n = theta.numel()
            assert all(k == n for k in plan.shape_sizes)
            gt = g.view(len(plan.shape_sizes), n).sum(0)
            return gt.to(theta.device, theta.dtype).view_as(theta)

    return _ShapeField.apply(theta)


# C-ABI names, for callers that want the flat interface.
def fresnel_last_error():
    return load_library().fresnel_last_error().decode()


def _spread_args(g1, g2, c, nf1, nf2, out):
    import torch
    for t in (g1, g2):
        assert t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()
    assert c.dtype == torch.complex64 and c.is_cuda and c.is_contiguous()
    n = g1.numel()
    assert g2.numel() == n and c.numel() == n
    if out is None:
        out = torch.empty((nf2, nf1), dtype=torch.complex64, device=g1.device)
    ptr = lambda t: t.data_ptr() if t.numel() > 0 else None
    return n, ptr(g1), ptr(g2), ptr(c), out


def fresnel_spread(g1, g2, c, nf1, nf2, w, beta, out=None, stream=None):
    """Spread N points (periodic grid coordinates g1, g2: float64 CUDA tensors;
    strengths c: complex64) onto an nf2 x nf1 complex64 grid with the
    exponential-of-semicircle kernel of width w and shape beta."""
    import torch
    n, p1, p2, pc, out = _spread_args(g1, g2, c, nf1, nf2, out)
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load_library().fresnel_spread(p1, p2, pc, n, int(nf1), int(nf2), int(w), float(beta),
                                         out.data_ptr(), ctypes.c_void_p(stream.cuda_stream)))
    return out


def fresnel_spread_noalloc(g1, g2, c, nf1, nf2, w, beta, out, stream=None):
    """fresnel_spread without any device allocation (for callers that cannot
    allocate): scratch is the library's static device array, so the caller
    must pass the output grid and keep calls on one device from overlapping."""
    import torch
    n, p1, p2, pc, out = _spread_args(g1, g2, c, nf1, nf2, out)
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load_library().fresnel_spread_noalloc(p1, p2, pc, n, int(nf1), int(nf2), int(w),
                                                 float(beta), out.data_ptr(),
                                                 ctypes.c_void_p(stream.cuda_stream)))
    return out
