"""Python binding of the TT-IGA C library (include/tt_iga.h).

Argument marshalling only: every step of geometry, assembly, solve and
evaluation runs in the CUDA kernels of libtt_iga.so.  PyTorch supplies device
memory (for the kernel-level calls and evaluation points) and the CUDA stream.
The functions keep the C names; failures raise TTIgaError carrying the status
code and the library's last error message.  There is no fallback: if the
shared library is missing, importing this package raises ImportError.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtt_iga.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libtt_iga.so is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_TOO_LARGE, ERR_BAD_GEOMETRY, ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
GEOM_BOX, GEOM_ANNULUS, GEOM_NURBS = 0, 1, 2
RHS_MANUFACTURED, RHS_CONSTANT, RHS_RING_LOG = 0, 1, 2
FP64, MIXED_FP32, MIXED_TF32 = 0, 1, 2
RHS_BLOCK, RHS_EACH = 0, 1
MAX_MODES = 8

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int_p = ctypes.POINTER(ctypes.c_int)


class TTIgaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tt_iga error {code}: {msg}")
        self.code = code


class CtxOpts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("alloc_fn", ctypes.c_void_p), ("free_fn", ctypes.c_void_p), ("alloc_user", ctypes.c_void_p)]


class GeomDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
                ("height", ctypes.c_double), ("twist", ctypes.c_double), ("swell", ctypes.c_double),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("p", ctypes.c_int), ("n", ctypes.c_int * 3), ("nq", ctypes.c_int),
                ("cross_tol", ctypes.c_double), ("max_rank", ctypes.c_int), ("seed", ctypes.c_uint64)]


class BcDesc(ctypes.Structure):
    _fields_ = [("dirichlet", ctypes.c_int * 6), ("value", ctypes.c_double * 6), ("flux", ctypes.c_double * 6)]


class NurbsPatch(ctypes.Structure):
    _fields_ = [("deg", ctypes.c_int * 3), ("ncp", ctypes.c_int * 3), ("knots", _c_double_p * 3),
                ("ctrl", _c_double_p), ("weights", _c_double_p)]


class RhsDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_modes", ctypes.c_int), ("a", ctypes.c_double * MAX_MODES),
                ("b", (ctypes.c_double * 3) * MAX_MODES), ("c", ctypes.c_double * MAX_MODES),
                ("value", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("precision", ctypes.c_int), ("max_sweeps", ctypes.c_int),
                ("kickrank", ctypes.c_int), ("max_rank", ctypes.c_int), ("local_maxit", ctypes.c_int),
                ("rhs_index", ctypes.c_int), ("verbose", ctypes.c_int), ("local_rtol", ctypes.c_double)]


class BatchItem(ctypes.Structure):
    _fields_ = [("geom", GeomDesc), ("n_rhs", ctypes.c_int), ("rhs", ctypes.POINTER(RhsDesc)),
                ("round_tol", ctypes.c_double), ("opts", SolveOpts), ("rhs_solve", ctypes.c_int),
                ("cores_out", _c_double_p), ("cores_cap", ctypes.c_size_t)]


class BatchResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("ranks", ctypes.c_int * 2), ("sweeps", ctypes.c_int),
                ("rel_residual_max", ctypes.c_double), ("dofs", ctypes.c_longlong), ("ms_geometry", ctypes.c_double),
                ("ms_assemble", ctypes.c_double), ("ms_solve", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_end_ms", ctypes.c_double), ("rhs_ranks", (ctypes.c_int * 2) * 8)]

    def as_dict(self):
        d = {k: (list(getattr(self, k)) if k == "ranks" else getattr(self, k)) for k, _ in self._fields_}
        d["rhs_ranks"] = [[self.rhs_ranks[k][0], self.rhs_ranks[k][1]] for k in range(8)]
        return d


class Stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("ranks", ctypes.c_int * 2), ("rel_residual", ctypes.c_double),
                ("local_residual", ctypes.c_double), ("local_matvecs", ctypes.c_longlong),
                ("local_matvecs_fp64", ctypes.c_longlong), ("ms_total", ctypes.c_double),
                ("converged", ctypes.c_int), ("local_matvecs_tensor", ctypes.c_longlong)]

    def as_dict(self):
        return {"sweeps": self.sweeps, "ranks": [self.ranks[0], self.ranks[1]],
                "rel_residual": self.rel_residual, "local_residual": self.local_residual,
                "local_matvecs": self.local_matvecs, "local_matvecs_fp64": self.local_matvecs_fp64,
                "local_matvecs_tensor": self.local_matvecs_tensor,
                "ms_total": self.ms_total, "converged": bool(self.converged)}


_vp = ctypes.c_void_p
_SIGS = {
    "tt_iga_ctx_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(CtxOpts)]),
    "tt_iga_ctx_destroy": (None, [_vp]),
    "tt_iga_last_error": (ctypes.c_char_p, [_vp]),
    "tt_iga_ctx_memory": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "tt_iga_launch_count": (ctypes.c_ulonglong, []),
    "tt_iga_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "tt_iga_profile_read": (ctypes.c_int, [_vp, _c_double_p, ctypes.POINTER(ctypes.c_longlong), _c_double_p]),
    "tt_iga_solution_cores": (ctypes.c_int, [_vp, _vp, _c_double_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int * 3),
                                             ctypes.POINTER(ctypes.c_int * 4)]),
    "tt_iga_geometry": (ctypes.c_int, [_vp, ctypes.POINTER(GeomDesc), ctypes.POINTER(_vp)]),
    "tt_iga_geom_destroy": (None, [_vp]),
    "tt_iga_geom_ranks": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int * 2 * 6), ctypes.POINTER(ctypes.c_double * 6)]),
    "tt_iga_geometry_nurbs": (ctypes.c_int, [_vp, ctypes.POINTER(GeomDesc), ctypes.POINTER(NurbsPatch),
                                             ctypes.POINTER(_vp)]),
    "tt_iga_assemble_bc": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(RhsDesc), ctypes.c_int, ctypes.c_double,
                                          ctypes.POINTER(BcDesc), ctypes.POINTER(_vp)]),
    "tt_iga_assemble": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(RhsDesc), ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(_vp)]),
    "tt_iga_system_destroy": (None, [_vp]),
    "tt_iga_system_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int * 2), ctypes.c_int, _vp,
                                          ctypes.POINTER(ctypes.c_int * 3)]),
    "tt_iga_solve": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(_vp), ctypes.POINTER(Stats)]),
    "tt_iga_system_stack": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_vp),
                                           _c_double_p]),
    "tt_iga_solution_unstack": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_vp)]),
    "tt_iga_solve_block": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(SolveOpts), ctypes.c_int, ctypes.POINTER(_vp),
                                          ctypes.POINTER(Stats), _c_double_p]),
    "tt_iga_solve_from": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(SolveOpts), _vp, ctypes.POINTER(_vp),
                                         ctypes.POINTER(Stats)]),
    "tt_iga_import_cores": (ctypes.c_int, [_vp, _vp, _c_double_p, ctypes.POINTER(ctypes.c_int * 3),
                                           ctypes.POINTER(ctypes.c_int * 4), ctypes.POINTER(_vp)]),
    "tt_iga_l2_diff": (ctypes.c_int, [_vp, _vp, _vp, _vp, _c_double_p]),
    "tt_iga_solution_destroy": (None, [_vp]),
    "tt_iga_solution_ranks": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int * 2)]),
    "tt_iga_residual": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _c_double_p]),
    "tt_iga_eval": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    "tt_iga_l2_error": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(RhsDesc), _c_double_p]),
    "tt_iga_densify_operator": (ctypes.c_int, [_vp, _vp, _c_double_p, ctypes.c_size_t]),
    "tt_iga_densify_rhs": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _c_double_p, ctypes.c_size_t]),
    "tt_iga_densify_solution": (ctypes.c_int, [_vp, _vp, _c_double_p, ctypes.c_size_t]),
    "tt_iga_operator_entries": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _c_int_p, _c_int_p, _c_double_p]),
    "tt_iga_vector_entries": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _c_int_p, _c_double_p]),
    "tt_iga_batch_solve": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(BatchItem), ctypes.c_int,
                                          ctypes.c_int, ctypes.POINTER(BatchResult), _c_double_p]),
    "tt_iga_batch_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(BatchItem), _c_int_p,
                                             ctypes.c_int, _c_int_p, ctypes.c_int, ctypes.POINTER(BatchResult),
                                             _c_int_p, _c_int_p, _c_double_p]),
    "tt_iga_ctx_set_sm_limit": (ctypes.c_int, [_vp, ctypes.c_int]),
    "tt_iga_basis_tables": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]),
    "tt_iga_geom_points": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(RhsDesc), ctypes.c_int, _vp, _vp,
                                          ctypes.POINTER(ctypes.c_longlong)]),
    "tt_iga_stiffness_core": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    "tt_iga_load_core": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int,
                                        ctypes.c_int, _vp]),
    "tt_iga_round": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int * 3), ctypes.POINTER(ctypes.c_int * 4),
                                    ctypes.POINTER(_vp * 3), ctypes.c_double, ctypes.c_int, ctypes.POINTER(_vp * 3),
                                    ctypes.POINTER(ctypes.c_int * 4)]),
    "tt_iga_gemm_f64": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_double, _vp,
                                       ctypes.c_int]),
    "tt_iga_qr": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp]),
    "tt_iga_svd_small": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp]),
    "tt_iga_blockband_solve": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]),
    "tt_iga_svd_small_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]),
    "tt_iga_maxvol": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_double, ctypes.c_int, _vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def exported_symbols():
    """Names of the C entry points this binding wraps."""
    return sorted(_SIGS)


def _check(ctx, code, allow=()):
    if code != OK and code not in allow:
        msg = _lib.tt_iga_last_error(ctx).decode() if ctx else ""
        raise TTIgaError(code, msg)
    return code


def _ptr(t):
    """Raw device pointer of a torch tensor (None -> NULL)."""
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ descriptors

def geom_desc(geometry, p, n, cross_tol=1e-10, max_rank=0, seed=0, nq=0):
    """GeomDesc from a geometry dict (see synthetic.py) and discretisation sizes."""
    d = GeomDesc()
    if geometry["kind"] == "annulus":
        d.kind = GEOM_ANNULUS
        d.r_in, d.r_out, d.height = geometry["r_in"], geometry["r_out"], geometry["height"]
        d.twist, d.swell = geometry.get("twist", 0.0), geometry.get("swell", 0.0)
    elif geometry["kind"] == "box":
        d.kind = GEOM_BOX
        d.lx, d.ly, d.lz = geometry["lx"], geometry["ly"], geometry["lz"]
    elif geometry["kind"] == "nurbs":
        d.kind = GEOM_NURBS  # the patch itself goes to tt_iga_geometry_nurbs
    else:
        raise ValueError("unknown geometry kind")
    d.p = int(p)
    nn = [int(n)] * 3 if isinstance(n, int) else [int(v) for v in n]
    for k in range(3):
        d.n[k] = nn[k]
    d.nq = int(nq)
    d.cross_tol = float(cross_tol)
    d.max_rank = int(max_rank)
    d.seed = int(seed)
    return d


def rhs_desc(modes=(), constant=None, ring_log=False):
    """RhsDesc: manufactured source with modulation modes [(a, (b1,b2,b3), c)], a constant f, or
    (ring_log) f = 0 whose exact solution is the log profile of the ring problem."""
    r = RhsDesc()
    if ring_log:
        r.kind = RHS_RING_LOG
        r.value = 0.0
        return r
    if constant is not None:
        r.kind = RHS_CONSTANT
        r.value = float(constant)
        return r
    modes = list(modes)
    if len(modes) > MAX_MODES:
        raise ValueError("too many modes")
    r.kind = RHS_MANUFACTURED
    r.n_modes = len(modes)
    for k, (a, b, c) in enumerate(modes):
        r.a[k] = a
        for j in range(3):
            r.b[k][j] = b[j]
        r.c[k] = c
    return r


def solve_opts(tol=1e-8, precision=FP64, max_sweeps=0, kickrank=0, max_rank=0, local_maxit=0, rhs_index=0,
               verbose=False, local_rtol=0.0):
    o = SolveOpts()
    o.tol, o.precision, o.max_sweeps, o.kickrank = tol, precision, max_sweeps, kickrank
    o.max_rank, o.local_maxit, o.rhs_index, o.verbose = max_rank, local_maxit, rhs_index, int(verbose)
    o.local_rtol = float(local_rtol)
    return o


# --------------------------------------------------------------------- calls

def tt_iga_ctx_create(stream=None, device=0):
    """Context on `device`, running on `stream` (a torch.cuda.Stream, a raw handle, or None)."""
    o = CtxOpts()
    if stream is not None:
        h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        # handle 0 is the legacy default stream; pass it as cudaStreamLegacy so the
        # library orders its work with the caller's instead of creating its own stream
        o.stream = h if h != 0 else 1
    o.device = device
    h = ctypes.c_void_p()
    _check(None, _lib.tt_iga_ctx_create(ctypes.byref(h), ctypes.byref(o)))
    return h


def tt_iga_ctx_destroy(ctx):
    _lib.tt_iga_ctx_destroy(ctx)


def tt_iga_last_error(ctx):
    return _lib.tt_iga_last_error(ctx).decode()


def tt_iga_ctx_memory(ctx):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(ctx, _lib.tt_iga_ctx_memory(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def tt_iga_launch_count():
    return int(_lib.tt_iga_launch_count())


PROF_OFF, PROF_LOCAL_BAND, PROF_GEMM64, PROF_QR = 0, 1, 2, 3


def tt_iga_profile_enable(ctx, family):
    _check(ctx, _lib.tt_iga_profile_enable(ctx, int(family)))


def tt_iga_profile_read(ctx):
    ms, n, w = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
    _check(ctx, _lib.tt_iga_profile_read(ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
    return ms.value, n.value, w.value


def tt_iga_solution_cores(ctx, u, out=None):
    """Solution TT cores copied to host. With out (a float64 numpy buffer, ideally pinned) fills it in place."""
    import numpy as np
    modes, ranks = (ctypes.c_int * 3)(), (ctypes.c_int * 4)()
    _check(ctx, _lib.tt_iga_solution_cores(ctx, u, None, 0, ctypes.byref(modes), ctypes.byref(ranks)))
    m, r = list(modes), list(ranks)
    sizes = [r[k] * m[k] * r[k + 1] for k in range(3)]
    tot = sum(sizes)
    if out is None:
        out = np.zeros(tot)
    _check(ctx, _lib.tt_iga_solution_cores(ctx, u, out.ctypes.data_as(_c_double_p), out.size, ctypes.byref(modes),
                                           ctypes.byref(ranks)))
    cores, off = [], 0
    for k in range(3):
        cores.append(out[off:off + sizes[k]].reshape(r[k], m[k], r[k + 1]))
        off += sizes[k]
    return cores


def tt_iga_geometry_nurbs(ctx, desc, degrees, knots, ctrl, weights, allow_not_converged=False):
    """Geometry on a NURBS patch: degrees (3), knots (3 arrays), ctrl [c1, c2, c3, 3] and
    weights [c1, c2, c3] with the xi_1 index first (numpy layout); desc.kind must be GEOM_NURBS."""
    import numpy as np
    ctrl = np.asarray(ctrl, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    c_fast = np.ascontiguousarray(ctrl.transpose(2, 1, 0, 3))  # xi_1 fastest, as the C ABI wants
    w_fast = np.ascontiguousarray(w.transpose(2, 1, 0))
    kn = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
    patch = NurbsPatch()
    for d in range(3):
        patch.deg[d] = int(degrees[d])
        patch.ncp[d] = int(ctrl.shape[d])
        patch.knots[d] = kn[d].ctypes.data_as(_c_double_p)
    patch.ctrl = c_fast.ctypes.data_as(_c_double_p)
    patch.weights = w_fast.ctypes.data_as(_c_double_p)
    h = ctypes.c_void_p()
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    code = _lib.tt_iga_geometry_nurbs(ctx, ctypes.byref(desc), ctypes.byref(patch), ctypes.byref(h))
    if code != OK and h.value and code not in allow:
        msg = tt_iga_last_error(ctx)
        _lib.tt_iga_geom_destroy(h)
        raise TTIgaError(code, msg)
    _check(ctx, code, allow)
    return h


def tt_iga_geometry(ctx, desc, allow_not_converged=False):
    h = ctypes.c_void_p()
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    code = _lib.tt_iga_geometry(ctx, ctypes.byref(desc), ctypes.byref(h))
    if code != OK and h.value:
        if code not in allow:
            msg = tt_iga_last_error(ctx)
            _lib.tt_iga_geom_destroy(h)
            raise TTIgaError(code, msg)
    else:
        _check(ctx, code, allow)
    return h


def tt_iga_geom_destroy(g):
    _lib.tt_iga_geom_destroy(g)


def tt_iga_geom_ranks(g):
    ranks = (ctypes.c_int * 2 * 6)()
    err = (ctypes.c_double * 6)()
    _check(None, _lib.tt_iga_geom_ranks(g, ctypes.byref(ranks), ctypes.byref(err)))
    return [(ranks[f][0], ranks[f][1]) for f in range(6)], list(err)


def tt_iga_assemble(ctx, g, rhs_list, round_tol=1e-12):
    arr = (RhsDesc * len(rhs_list))(*rhs_list)
    h = ctypes.c_void_p()
    _check(ctx, _lib.tt_iga_assemble(ctx, g, arr, len(rhs_list), round_tol, ctypes.byref(h)))
    return h


def bc_desc(dirichlet, values=(0.0,) * 6, flux=(0.0,) * 6):
    """BcDesc: dirichlet[f] (bool), constant value[f] (Dirichlet faces) and constant outward
    normal flux[f] (natural faces) for face f = 2 d + side."""
    b = BcDesc()
    for f in range(6):
        b.dirichlet[f] = 1 if dirichlet[f] else 0
        b.value[f] = float(values[f])
        b.flux[f] = float(flux[f])
    return b


def tt_iga_assemble_bc(ctx, g, rhs_list, bc, round_tol=1e-12):
    arr = (RhsDesc * len(rhs_list))(*rhs_list)
    h = ctypes.c_void_p()
    _check(ctx, _lib.tt_iga_assemble_bc(ctx, g, arr, len(rhs_list), round_tol, ctypes.byref(bc), ctypes.byref(h)))
    return h


def tt_iga_system_destroy(s):
    _lib.tt_iga_system_destroy(s)


def tt_iga_system_info(s, n_rhs_max=8):
    op = (ctypes.c_int * 2)()
    rr = (ctypes.c_int * 2 * n_rhs_max)()
    modes = (ctypes.c_int * 3)()
    cnt = _lib.tt_iga_system_info(s, ctypes.byref(op), n_rhs_max, ctypes.cast(rr, ctypes.c_void_p), ctypes.byref(modes))
    if cnt < 0:
        raise TTIgaError(cnt, "system_info")
    return {"op_ranks": (op[0], op[1]), "rhs_ranks": [(rr[k][0], rr[k][1]) for k in range(min(cnt, n_rhs_max))],
            "modes": (modes[0], modes[1], modes[2]), "n_rhs": cnt}


def tt_iga_solve(ctx, s, opts, allow_not_converged=False):
    h = ctypes.c_void_p()
    st = Stats()
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    code = _lib.tt_iga_solve(ctx, s, ctypes.byref(opts), ctypes.byref(h), ctypes.byref(st))
    if code != OK and code not in allow:
        msg = tt_iga_last_error(ctx)
        if h.value:
            _lib.tt_iga_solution_destroy(h)
        raise TTIgaError(code, msg)
    return h, st.as_dict()


def tt_iga_solution_destroy(u):
    _lib.tt_iga_solution_destroy(u)


def tt_iga_solve_from(ctx, s, opts, u0, allow_not_converged=False):
    """AMEn solve of s started from the iterate u0 (a solution handle); returns (handle, stats)."""
    h = ctypes.c_void_p()
    st = Stats()
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    code = _lib.tt_iga_solve_from(ctx, s, ctypes.byref(opts), u0, ctypes.byref(h), ctypes.byref(st))
    if code != OK and code not in allow:
        msg = tt_iga_last_error(ctx)
        if h.value:
            _lib.tt_iga_solution_destroy(h)
        raise TTIgaError(code, msg)
    return h, st.as_dict()


def tt_iga_import_cores(ctx, s, cores):
    """Solution of system s from host TT cores (three float64 arrays [r0, m, r1], as returned by
    tt_iga_solution_cores)."""
    import numpy as np
    cores = [np.ascontiguousarray(c, dtype=np.float64) for c in cores]
    modes = (ctypes.c_int * 3)(*[int(c.shape[1]) for c in cores])
    ranks = (ctypes.c_int * 4)(int(cores[0].shape[0]), int(cores[0].shape[2]), int(cores[1].shape[2]),
                               int(cores[2].shape[2]))
    flat = np.concatenate([c.reshape(-1) for c in cores])
    h = ctypes.c_void_p()
    _check(ctx, _lib.tt_iga_import_cores(ctx, s, flat.ctypes.data_as(_c_double_p), ctypes.byref(modes),
                                         ctypes.byref(ranks), ctypes.byref(h)))
    return h


def tt_iga_l2_diff(ctx, g, u, v):
    """Relative L2 difference ||u_h - v_h|| / ||v_h|| over the mapped domain of g."""
    r = ctypes.c_double()
    _check(ctx, _lib.tt_iga_l2_diff(ctx, g, u, v, ctypes.byref(r)))
    return r.value


def tt_iga_system_stack(ctx, s, mode=1, eps=0.0):
    """Block system of all right-hand sides of s merged into TT mode `mode`; returns (handle, [||F_k||])."""
    nrhs = tt_iga_system_info(s)["n_rhs"]
    h = ctypes.c_void_p()
    sc = (ctypes.c_double * nrhs)()
    _check(ctx, _lib.tt_iga_system_stack(ctx, s, mode, eps, ctypes.byref(h), sc))
    return h, list(sc)


def tt_iga_solution_unstack(ctx, ub, k, scale):
    h = ctypes.c_void_p()
    _check(ctx, _lib.tt_iga_solution_unstack(ctx, ub, k, scale, ctypes.byref(h)))
    return h


def tt_iga_solve_block(ctx, s, opts, mode=-1, allow_not_converged=False):
    """One block-TT solve of every right-hand side of s; returns ([solutions], stats, [rel. residuals])."""
    nrhs = tt_iga_system_info(s)["n_rhs"]
    hs = (_vp * nrhs)()
    st = Stats()
    rr = (ctypes.c_double * nrhs)()
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    code = _lib.tt_iga_solve_block(ctx, s, ctypes.byref(opts), mode, hs, ctypes.byref(st), rr)
    sols = [ctypes.c_void_p(h) for h in hs]
    if code != OK and code not in allow:
        msg = tt_iga_last_error(ctx)
        for h in sols:
            if h.value:
                _lib.tt_iga_solution_destroy(h)
        raise TTIgaError(code, msg)
    return sols, st.as_dict(), list(rr)


def tt_iga_solution_ranks(u):
    r = (ctypes.c_int * 2)()
    _check(None, _lib.tt_iga_solution_ranks(u, ctypes.byref(r)))
    return r[0], r[1]


def tt_iga_residual(ctx, s, u, k=0):
    v = ctypes.c_double()
    _check(ctx, _lib.tt_iga_residual(ctx, s, u, k, ctypes.byref(v)))
    return v.value


def tt_iga_eval(ctx, u, xi, out):
    """u_h at parametric points xi (torch float64 CUDA tensor [m, 3]) into out (float64 CUDA [m])."""
    _check(ctx, _lib.tt_iga_eval(ctx, u, int(xi.shape[0]), _ptr(xi), _ptr(out)))
    return out


def tt_iga_l2_error(ctx, g, u, rhs):
    v = ctypes.c_double()
    _check(ctx, _lib.tt_iga_l2_error(ctx, g, u, ctypes.byref(rhs), ctypes.byref(v)))
    return v.value


def _host_buffer(n):
    import numpy as np
    a = np.zeros(n, dtype=np.float64)
    return a, a.ctypes.data_as(_c_double_p)


def tt_iga_densify_operator(ctx, s):
    import numpy as np
    m = tt_iga_system_info(s)["modes"]
    N = m[0] * m[1] * m[2]
    a, p = _host_buffer(N * N)
    _check(ctx, _lib.tt_iga_densify_operator(ctx, s, p, N * N))
    return a.reshape(N, N)


def tt_iga_densify_rhs(ctx, s, k=0):
    m = tt_iga_system_info(s)["modes"]
    N = m[0] * m[1] * m[2]
    a, p = _host_buffer(N)
    _check(ctx, _lib.tt_iga_densify_rhs(ctx, s, k, p, N))
    return a


def tt_iga_densify_solution(ctx, u, modes):
    N = modes[0] * modes[1] * modes[2]
    a, p = _host_buffer(N)
    _check(ctx, _lib.tt_iga_densify_solution(ctx, u, p, N))
    return a


def tt_iga_operator_entries(ctx, s, rows, cols):
    import numpy as np
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros(len(rows))
    _check(ctx, _lib.tt_iga_operator_entries(ctx, s, len(rows), rows.ctypes.data_as(_c_int_p),
                                             cols.ctypes.data_as(_c_int_p), out.ctypes.data_as(_c_double_p)))
    return out


def tt_iga_vector_entries(ctx, s, u, k, idx):
    import numpy as np
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.zeros(len(idx))
    _check(ctx, _lib.tt_iga_vector_entries(ctx, s, u, k, len(idx), idx.ctypes.data_as(_c_int_p),
                                           out.ctypes.data_as(_c_double_p)))
    return out


def batch_items(instances, tol=1e-8, precision=FP64, cross_tol=1e-10, round_tol=1e-12, max_rank=0,
                rhs_solve=None, cores_cap=0):
    """BatchItem array from instance dicts (synthetic.random_instance); keeps the rhs arrays alive.
    rhs_solve: RHS_BLOCK (default) or RHS_EACH.  cores_cap > 0: every item gets a host buffer of that
    many doubles for its solutions' cores (keep[1][k] is item k's numpy buffer)."""
    arr = (BatchItem * len(instances))()
    keep = []
    for k, inst in enumerate(instances):
        arr[k].geom = geom_desc(inst["geometry"], inst["p"], inst["n"], cross_tol=cross_tol, seed=inst.get("seed", 0),
                                max_rank=max_rank)
        rh = (RhsDesc * len(inst["rhs"]))(*[rhs_desc(m) for m in inst["rhs"]])
        keep.append(rh)
        arr[k].n_rhs = len(inst["rhs"])
        arr[k].rhs = ctypes.cast(rh, ctypes.POINTER(RhsDesc))
        arr[k].round_tol = round_tol
        arr[k].opts = solve_opts(tol=tol, precision=precision)
        arr[k].rhs_solve = RHS_BLOCK if rhs_solve is None else int(rhs_solve)
    bufs = []
    if cores_cap > 0:
        import numpy as np
        for k in range(len(instances)):
            b = np.zeros(int(cores_cap))
            bufs.append(b)
            arr[k].cores_out = b.ctypes.data_as(_c_double_p)
            arr[k].cores_cap = int(cores_cap)
    return arr, (keep, bufs)


def batch_cores(item_buf, result, n):
    """Split an item's cores buffer into [rhs][3 cores] with the result's ranks (unknowns n - 2)."""
    m = n - 2
    out, off = [], 0
    for k in range(8):
        r1, r2 = result["rhs_ranks"][k]
        if r1 == 0:
            break
        sizes = [(1, m, r1), (r1, m, r2), (r2, m, 1)]
        cores = []
        for sh in sizes:
            cnt = sh[0] * sh[1] * sh[2]
            cores.append(item_buf[off:off + cnt].reshape(sh))
            off += cnt
        out.append(cores)
    return out


def tt_iga_batch_solve(items, lanes, device=0, sm_per_lane=-1):
    """Returns (status, per-instance result dicts, wall ms).  sm_per_lane: -1 an equal SM share per
    lane, 0 the whole GPU for every lane, > 0 that many SMs."""
    n = len(items)
    res = (BatchResult * max(1, n))()
    ms = ctypes.c_double()
    code = _lib.tt_iga_batch_solve(device, n, items, lanes, sm_per_lane, res, ctypes.byref(ms))
    return code, [res[i].as_dict() for i in range(n)], ms.value


def tt_iga_batch_autotune(items, candidates, device=0, shares=(-1,)):
    """Fastest (lanes, sm_per_lane) pair over candidates x shares; returns (lanes, sm_per_lane, ms, results)."""
    n = len(items)
    res = (BatchResult * max(1, n))()
    cand = (ctypes.c_int * len(candidates))(*candidates)
    sh = (ctypes.c_int * len(shares))(*shares)
    best, best_share, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    code = _lib.tt_iga_batch_autotune(device, n, items, cand, len(candidates), sh, len(shares), res,
                                      ctypes.byref(best), ctypes.byref(best_share), ctypes.byref(ms))
    _check(None, code, (ERR_NOT_CONVERGED,))
    return best.value, best_share.value, ms.value, [res[i].as_dict() for i in range(n)]


def tt_iga_ctx_set_sm_limit(ctx, max_sms):
    _check(ctx, _lib.tt_iga_ctx_set_sm_limit(ctx, int(max_sms)))


def tt_iga_basis_tables(ctx, n, p, nq, pts, wts, N, dN):
    _check(ctx, _lib.tt_iga_basis_tables(ctx, n, p, nq, _ptr(pts), _ptr(wts), _ptr(N), _ptr(dN)))


def tt_iga_geom_points(ctx, g, rhs, idx, out):
    bad = ctypes.c_longlong()
    _check(ctx, _lib.tt_iga_geom_points(ctx, g, ctypes.byref(rhs) if rhs is not None else None, int(idx.shape[0]),
                                        _ptr(idx), _ptr(out), ctypes.byref(bad)))
    return bad.value


def tt_iga_stiffness_core(ctx, n, p, nq, wts, N, dN, G, r0, r1, test_deriv, trial_deriv, M):
    _check(ctx, _lib.tt_iga_stiffness_core(ctx, n, p, nq, _ptr(wts), _ptr(N), _ptr(dN), _ptr(G), r0, r1,
                                           int(test_deriv), int(trial_deriv), _ptr(M)))


def tt_iga_load_core(ctx, n, p, nq, wts, N, G, r0, r1, F):
    _check(ctx, _lib.tt_iga_load_core(ctx, n, p, nq, _ptr(wts), _ptr(N), _ptr(G), r0, r1, _ptr(F)))


def tt_iga_round(ctx, cores, eps, max_rank=0):
    """Round a TT given as three float64 CUDA tensors [r0, m, r1]; returns (cores, ranks)."""
    import torch
    nm = (ctypes.c_int * 3)(*[int(G.shape[1]) for G in cores])
    r = (ctypes.c_int * 4)(1, int(cores[0].shape[2]), int(cores[1].shape[2]), 1)
    cin = (ctypes.c_void_p * 3)(*[G.data_ptr() for G in cores])
    outs = [torch.empty_like(G) for G in cores]
    cout = (ctypes.c_void_p * 3)(*[t.data_ptr() for t in outs])
    rout = (ctypes.c_int * 4)()
    _check(ctx, _lib.tt_iga_round(ctx, ctypes.byref(nm), ctypes.byref(r), ctypes.byref(cin), eps, max_rank,
                                  ctypes.byref(cout), ctypes.byref(rout)))
    res = []
    for k in range(3):
        cnt = rout[k] * nm[k] * rout[k + 1]
        res.append(outs[k].reshape(-1)[:cnt].reshape(rout[k], nm[k], rout[k + 1]))
    return res, [rout[k] for k in range(4)]


def tt_iga_gemm_f64(ctx, ta, tb, alpha, A, B, beta, C):
    """C = alpha op(A) op(B) + beta C on float64 CUDA tensors (row-major, contiguous)."""
    m, n = int(C.shape[0]), int(C.shape[1])
    k = int(A.shape[0] if ta else A.shape[1])
    _check(ctx, _lib.tt_iga_gemm_f64(ctx, int(ta), int(tb), m, n, k, alpha, _ptr(A), int(A.stride(0)), _ptr(B),
                                     int(B.stride(0)), beta, _ptr(C), int(C.stride(0))))


def tt_iga_qr(ctx, A, Q, R):
    m, k = int(A.shape[0]), int(A.shape[1])
    _check(ctx, _lib.tt_iga_qr(ctx, m, k, _ptr(A), int(A.stride(0)), _ptr(Q), _ptr(R)))


def tt_iga_svd_small(ctx, A, U, s, V):
    _check(ctx, _lib.tt_iga_svd_small(ctx, int(A.shape[0]), _ptr(A), _ptr(U), _ptr(s), _ptr(V)))


def tt_iga_blockband_solve(ctx, PhiL, A, PhiR, r, z):
    """z = B^{-1} r with the block-band preconditioner of the local system B = sym(PhiL (x) A (x) PhiR)
    (device tensors: PhiL [rl][Rl][rl], A [Rl][n][2p+1][Rr] band-stored, PhiR [rr][Rr][rr], r and z [rl*n*rr])."""
    rl, Rl = int(PhiL.shape[0]), int(PhiL.shape[1])
    rr, Rr = int(PhiR.shape[0]), int(PhiR.shape[1])
    n, p = int(A.shape[1]), (int(A.shape[2]) - 1) // 2
    _check(ctx, _lib.tt_iga_blockband_solve(ctx, rl, rr, Rl, Rr, n, p, _ptr(PhiL), _ptr(A), _ptr(PhiR), _ptr(r),
                                            _ptr(z)))


def tt_iga_svd_small_noalloc(stream, A, U, s, V, info=None):
    """Allocation-free SVD on `stream` (torch.cuda.Stream, raw handle or None for the legacy default stream).

    info: optional int32 CUDA tensor of one element, set to 0 (converged) or 1 (not converged).
    Returns the status code instead of raising, so callers can see ERR_TOO_LARGE for k > 256."""
    h = None
    if stream is not None:
        h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return int(_lib.tt_iga_svd_small_noalloc(h, int(A.shape[0]), _ptr(A), _ptr(U), _ptr(s), _ptr(V), _ptr(info)))


def tt_iga_maxvol(ctx, U, rows, B, delta=1e-2, maxit=100):
    _check(ctx, _lib.tt_iga_maxvol(ctx, int(U.shape[0]), int(U.shape[1]), _ptr(U), delta, maxit, _ptr(rows), _ptr(B)))
