"""ctypes binding of liblsms (include/lsms.h): argument marshalling only.

Every computation happens in the CUDA library.  If the library is missing this module raises: there
is no CPU fallback.  Host arrays are NumPy complex128 (interleaved, the layout the ABI expects);
device entry points take torch tensors (complex128, CUDA) and a stream.

Context covers the C ABI: three-layer media (Context(k1, k2, k3, d, ...)) or any stack of layers,
absorbing ones included (stack=(ks, thicknesses, particle_layer), complex ks); particles or batches
of layouts (set_particles, set_layouts); dense rotated scattering matrices for inclusions of any
shape (set_scattering_matrix, set_orientations; inclusion_scattering_matrix,
pec_scattering_diagonal and, with a complex kp for absorbing particles, scattering_diagonal and
inclusion_scattering_matrix build them on the host); the translation through boxes (set_fmm); the
operator and its steps, solves and fields.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblsms.so")

LSMS_FP64, LSMS_MIXED = 0, 1
APPLY_SCALED, APPLY_MIXED, APPLY_NO_TRANSLATION, APPLY_NO_REFLECTION, APPLY_ALPHA = 1, 2, 4, 8, 16
FIELD_TOTAL, FIELD_SCATTERED, FIELD_PARTICLE = 0, 1, 2
FMM_ALL, FMM_RESIDUAL = 0, 1
STATUS = {0: "OK", -1: "ARG", -2: "GEOMETRY", -3: "NOT_CONVERGED", -4: "NONFINITE", -5: "OOM",
          -6: "CUDA", -7: "STATE"}
EXPORTS = ["lsms_create", "lsms_layer_response", "lsms_build_contour_stack", "lsms_pec_scattering_diagonal", "lsms_scattering_diagonal_c", "lsms_set_scattering_diagonal", "lsms_inclusion_scattering_matrix_c", "lsms_set_fmm", "lsms_set_fmm_scope", "lsms_get_fmm", "lsms_fmm_stats", "lsms_create_stack", "lsms_create_stack_c", "lsms_set_scattering_matrix", "lsms_set_orientations",
           "lsms_get_scattering_matrix", "lsms_inclusion_scattering_matrix", "lsms_set_particles", "lsms_apply", "lsms_apply_ex", "lsms_apply_dev", "lsms_apply_rows_dev",
           "lsms_translate", "lsms_aggregate", "lsms_reflect", "lsms_disaggregate", "lsms_incident",
           "lsms_get_contour", "lsms_get_scattering", "lsms_num_nodes", "lsms_num_particles",
           "lsms_solve", "lsms_eval_field", "lsms_last_error", "lsms_destroy",
           "lsms_build_contour", "lsms_scattering_diagonal", "lsms_check_geometry",
           "lsms_set_timing", "lsms_last_timing", "lsms_translate_mixed_noalloc",
           "lsms_set_layouts", "lsms_num_layouts", "lsms_autotune", "lsms_set_tc_translation",
           "lsms_get_translation_tuning", "lsms_set_translation_tuning", "lsms_get_batch_translation"]


class LsmsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lsms error {code} ({STATUS.get(code, '?')}): {msg}")
        self.code = code


class Contour(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int), ("b", ctypes.c_double), ("t_max", ctypes.c_double),
                ("panel_order", ctypes.c_int), ("panel_rule", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("rel_res_fp64", ctypes.c_double), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_cap", ctypes.c_int), ("n_history", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblsms.so (built by paper_1407_3868_gb300.build).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"liblsms.so not found at {path}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "lsms_create": (i, [d, d, d, d, d, d, i, ctypes.POINTER(Contour), i, ctypes.POINTER(_P)]),
        "lsms_create_stack": (i, [i, _D, _D, i, d, d, i, ctypes.POINTER(Contour), i, ctypes.POINTER(_P)]),
        "lsms_create_stack_c": (i, [i, _D, _D, i, d, d, i, ctypes.POINTER(Contour), i, ctypes.POINTER(_P)]),
        "lsms_set_particles": (i, [_P, i, _D]),
        "lsms_set_scattering_matrix": (i, [_P, _D]),
        "lsms_set_fmm": (i, [_P, d, i]),
        "lsms_set_fmm_scope": (i, [_P, i]),
        "lsms_get_fmm": (i, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "lsms_fmm_stats": (i, [_P, ctypes.POINTER(ctypes.c_longlong), _D, _D]),
        "lsms_set_orientations": (i, [_P, i, _D]),
        "lsms_get_scattering_matrix": (i, [_P, _D]),
        "lsms_inclusion_scattering_matrix": (i, [i, d, d, d, i, _D, _D]),
        "lsms_pec_scattering_diagonal": (i, [i, d, d, _D]),
        "lsms_scattering_diagonal_c": (i, [i, d, d, d, d, _D]),
        "lsms_set_scattering_diagonal": (i, [_P, _D]),
        "lsms_inclusion_scattering_matrix_c": (i, [i, d, d, d, d, i, _D, _D]),
        "lsms_apply": (i, [_P, i, _D, _D]),
        "lsms_apply_ex": (i, [_P, i, _D, _D, i]),
        "lsms_apply_dev": (i, [_P, i, _P, _P, i, _P]),
        "lsms_apply_rows_dev": (i, [_P, i, i, i, _P, _P, i, _P]),
        "lsms_translate": (i, [_P, i, _D, _D, i]),
        "lsms_aggregate": (i, [_P, i, _D, _D, _D, i]),
        "lsms_reflect": (i, [_P, i, _D, _D, _D, _D]),
        "lsms_disaggregate": (i, [_P, i, _D, _D, _D, i]),
        "lsms_incident": (i, [_P, i, _D, _D]),
        "lsms_get_contour": (i, [_P, _D, _D]),
        "lsms_get_scattering": (i, [_P, _D]),
        "lsms_num_nodes": (i, [_P]),
        "lsms_num_particles": (i, [_P]),
        "lsms_solve": (i, [_P, i, _D, d, i, _D, _D, ctypes.POINTER(SolveInfo)]),
        "lsms_eval_field": (i, [_P, i, i, _D, i, _D]),
        "lsms_last_error": (ctypes.c_char_p, [_P]),
        "lsms_destroy": (None, [_P]),
        "lsms_build_contour": (i, [ctypes.POINTER(Contour), d, d, d, _D, _D]),
        "lsms_build_contour_stack": (i, [ctypes.POINTER(Contour), i, _D, _D, _D]),
        "lsms_layer_response": (i, [i, _D, _D, i, i, _D, _D]),
        "lsms_scattering_diagonal": (i, [i, d, d, d, _D]),
        "lsms_check_geometry": (i, [d, d, i, _D]),
        "lsms_set_timing": (i, [_P, i]),
        "lsms_last_timing": (i, [_P, _D, _D, ctypes.POINTER(ctypes.c_int)]),
        "lsms_translate_mixed_noalloc": (i, [i, i, d, i, _P, _P, _P, _P]),
        "lsms_set_layouts": (i, [_P, i, ctypes.POINTER(ctypes.c_int), _D]),
        "lsms_num_layouts": (i, [_P]),
        "lsms_autotune": (i, [_P, _D]),
        "lsms_get_translation_tuning": (i, [_P, i, ctypes.POINTER(ctypes.c_int), _D]),
        "lsms_set_translation_tuning": (i, [_P, i, i, d]),
        "lsms_get_batch_translation": (i, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "lsms_set_tc_translation": (i, [_P, i, i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _c128(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Context:
    """One lsms context (lsms_create ... lsms_destroy)."""

    def __init__(self, k1, k2, k3, d, kp, radius, p, n_nodes, b=0.0, t_max=0.0, panel_order=0,
                 precision=LSMS_FP64, stack=None, panel_rule=0):
        """Three layers (k1, k2, k3; middle thickness d), or with stack=(ks, thicknesses, m) any
        number of layers (k1, k2, k3 and d are then ignored; lsms_create_stack, or with complex ks
        — absorbing layers — lsms_create_stack_c).  panel_rule: lsms_contour.panel_rule."""
        self.lib = load()
        self.p = p
        self.P = 2 * p + 1
        c = Contour(n_nodes, b, t_max, panel_order, panel_rule)
        h = _P()
        if stack is None:
            rc = self.lib.lsms_create(k1, k2, k3, d, kp, radius, p, ctypes.byref(c), precision,
                                      ctypes.byref(h))
        else:
            lossy = np.iscomplexobj(np.asarray(stack[0]))
            ks = np.ascontiguousarray(stack[0], dtype=np.complex128 if lossy else np.float64)
            ds = np.ascontiguousarray(stack[1], dtype=np.float64)
            if ds.size != max(ks.size - 2, 0):
                raise LsmsError(-1, "stack: need len(ks) - 2 thicknesses")
            create = self.lib.lsms_create_stack_c if lossy else self.lib.lsms_create_stack
            rc = create(int(ks.size), _dptr(ks), _dptr(ds), int(stack[2]), kp, radius, p, ctypes.byref(c),
                        precision, ctypes.byref(h))
        if rc != 0:
            raise LsmsError(rc, self.lib.lsms_last_error(None).decode())
        self.h = h
        self.n = -1
        self.ns = self.lib.lsms_num_nodes(h)

    # -- lifetime ------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.lsms_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc):
        if rc != 0:
            raise LsmsError(rc, self.lib.lsms_last_error(self.h).decode())
        return rc

    # -- setup -----------------------------------------------------------------------------------
    def set_particles(self, centres):
        c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 2)
        self._check(self.lib.lsms_set_particles(self.h, c.shape[0], _dptr(c)))
        self.n = c.shape[0]
        self.layout_counts = None

    def set_layouts(self, layouts):
        """A batch of independent layouts: `layouts` is a list of (N_l, 2) centre arrays."""
        counts = np.array([len(c) for c in layouts], dtype=np.int32)
        xy = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).reshape(-1, 2)
                                                  for c in layouts]) if len(layouts) else
                                  np.zeros((0, 2)))
        self._check(self.lib.lsms_set_layouts(self.h, len(layouts), counts.ctypes.data_as(
            ctypes.POINTER(ctypes.c_int)), _dptr(xy)))
        self.n = int(counts.sum())
        self.layout_counts = counts

    def autotune(self, cache=None):
        """lsms_autotune: the FP32 translation's tile shape (0: two lanes per target disc, 1: four
        lanes per target, 2: one Hankel sequence per unordered pair) and split factor per size
        bucket; for a batch, when timed, also the one-launch translation's kernel and coverage
        (batch_translation()).

        cache: path of a JSON file of earlier results, keyed by (p, contour nodes, power-of-two size
        bucket): when every layout's bucket is there the stored tuning is applied without timing
        (the batch's one-launch translation then keeps its defaults), otherwise the library times
        the candidates and the file is updated.  Returns the list of (shape, split multiplier) per
        layout."""
        import json
        counts = self.layout_counts if getattr(self, "layout_counts", None) is not None else [self.n]
        keys = [f"p{self.p}_ns{self.ns}_b{int(np.ceil(np.log2(n))) if n > 0 else 0}" for n in counts]
        table = {}
        if cache is not None and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        batch = getattr(self, "layout_counts", None) is not None
        if cache is not None and all(k in table for k in keys):
            for layout, k in enumerate(keys):
                self.set_translation_tuning(layout if batch else -1, table[k]["shape"], table[k]["split_mult"])
        else:
            m = ctypes.c_double()
            self._check(self.lib.lsms_autotune(self.h, ctypes.byref(m)))
        tuning = [self.translation_tuning(layout if batch else 0) for layout in range(len(counts))]
        if cache is not None:
            for k, (shape, mult) in zip(keys, tuning):
                table[k] = {"shape": shape, "split_mult": mult}
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return tuning

    def translation_tuning(self, layout=0):
        """lsms_get_translation_tuning: (tile shape, split multiplier) of a layout."""
        shape, mult = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.lsms_get_translation_tuning(self.h, int(layout), ctypes.byref(shape), ctypes.byref(mult)))
        return shape.value, mult.value

    def batch_translation(self):
        """lsms_get_batch_translation: (waves, work items) of a batch's one-launch translation."""
        waves, items = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.lsms_get_batch_translation(self.h, ctypes.byref(waves), ctypes.byref(items)))
        return waves.value, items.value

    def set_translation_tuning(self, layout, shape, split_mult):
        """lsms_set_translation_tuning (layout -1: every layout)."""
        self._check(self.lib.lsms_set_translation_tuning(self.h, int(layout), int(shape), float(split_mult)))

    def set_fmm(self, box_width: float, order: int = 0):
        """Translation through boxes of this width (0: all pairs); order 0 picks k2 r_box + 32."""
        self._check(self.lib.lsms_set_fmm(self.h, float(box_width), int(order)))

    def set_fmm_scope(self, scope: int):
        """lsms_set_fmm_scope: FMM_ALL (every translation) or FMM_RESIDUAL (only the FP64 residuals of
        the mixed refinement)."""
        self._check(self.lib.lsms_set_fmm_scope(self.h, int(scope)))

    def fmm_stats(self):
        """(directly translated pairs, far-part ms, near-part ms of the last timed translation)."""
        pairs, a, b = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.lsms_fmm_stats(self.h, ctypes.byref(pairs), ctypes.byref(a), ctypes.byref(b)))
        return pairs.value, a.value, b.value

    def fmm_info(self):
        nb, q = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.lsms_get_fmm(self.h, ctypes.byref(nb), ctypes.byref(q)))
        return nb.value, q.value

    def set_scattering_matrix(self, smat=None):
        """Dense prototype scattering matrix [P][P] (None: the disc's Mie diagonal)."""
        if smat is None:
            self._check(self.lib.lsms_set_scattering_matrix(self.h, None))
            return
        s = _c128(smat, (self.P, self.P))
        self._check(self.lib.lsms_set_scattering_matrix(self.h, _dptr(s)))

    def set_scattering_diagonal(self, s=None):
        """lsms_set_scattering_diagonal: S_n (2p + 1 complex) of every disc, or None for the Mie
        diagonal of the context's kp."""
        sd = None if s is None else _c128(s, (self.P,))
        self._check(self.lib.lsms_set_scattering_diagonal(self.h, _dptr(sd)))

    def set_orientations(self, theta=None):
        """Rotation angles of the particles (None: all zero)."""
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
        n = self.n if th is None else th.size
        self._check(self.lib.lsms_set_orientations(self.h, int(n), _dptr(th)))

    def scattering_matrix(self):
        s = np.zeros((self.P, self.P), dtype=np.complex128)
        self._check(self.lib.lsms_get_scattering_matrix(self.h, _dptr(s)))
        return s

    def set_tc_translation(self, min_rhs: int, flush: int = 0):
        """Blocks of at least min_rhs right-hand sides: mixed translation on the tensor cores (0 = never);
        flush: source discs per FP32 accumulation before draining into FP64 (0 = keep)."""
        self._check(self.lib.lsms_set_tc_translation(self.h, int(min_rhs), int(flush)))

    def contour(self):
        lam = np.zeros(self.ns, dtype=np.complex128)
        wt = np.zeros(self.ns, dtype=np.complex128)
        self._check(self.lib.lsms_get_contour(self.h, _dptr(lam), _dptr(wt)))
        return lam, wt

    def scattering(self):
        s = np.zeros(self.P, dtype=np.complex128)
        self._check(self.lib.lsms_get_scattering(self.h, _dptr(s)))
        return s

    # -- operator and its steps ------------------------------------------------------------------
    def _coeffs(self, x):
        x = _c128(x)
        nrhs = x.size // (self.n * self.P) if self.n > 0 else (x.shape[0] if x.ndim == 3 else 1)
        return _c128(x, (nrhs, self.n, self.P)), nrhs

    def apply(self, x, flags=0):
        x, nrhs = self._coeffs(x)
        y = np.zeros_like(x)
        self._check(self.lib.lsms_apply_ex(self.h, nrhs, _dptr(x), _dptr(y), flags))
        return y

    def apply_default(self, x):
        x, nrhs = self._coeffs(x)
        y = np.zeros_like(x)
        self._check(self.lib.lsms_apply(self.h, nrhs, _dptr(x), _dptr(y)))
        return y

    def apply_dev(self, x, y, flags=0, stream=None):
        """x, y: CUDA complex128 torch tensors of shape (nrhs, N, P); asynchronous on `stream`."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        nrhs = x.numel() // (self.n * self.P)
        self._check(self.lib.lsms_apply_dev(self.h, nrhs, ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(y.data_ptr()), flags,
                                            ctypes.c_void_p(stream.cuda_stream)))

    def apply_rows_dev(self, x, y, row0, row1, flags=0, stream=None):
        """lsms_apply_rows_dev: y (nrhs, row1 - row0, P) = rows row0 .. row1 - 1 of the operator applied
        to x (nrhs, N, P); CUDA complex128 tensors, asynchronous on `stream`."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        nrhs = x.numel() // (self.n * self.P) if self.n > 0 else 0
        if y.numel() != nrhs * (row1 - row0) * self.P:
            raise ValueError("apply_rows_dev: y must hold nrhs x (row1 - row0) x P values")
        self._check(self.lib.lsms_apply_rows_dev(self.h, nrhs, int(row0), int(row1), ctypes.c_void_p(x.data_ptr()),
                                                 ctypes.c_void_p(y.data_ptr()), flags,
                                                 ctypes.c_void_p(stream.cuda_stream)))

    def translate(self, beta, precision=LSMS_FP64):
        x, nrhs = self._coeffs(beta)
        a = np.zeros_like(x)
        self._check(self.lib.lsms_translate(self.h, nrhs, _dptr(x), _dptr(a), precision))
        return a

    def aggregate(self, beta, precision=LSMS_FP64):
        x, nrhs = self._coeffs(beta)
        pp = np.zeros((nrhs, self.ns), dtype=np.complex128)
        qm = np.zeros_like(pp)
        self._check(self.lib.lsms_aggregate(self.h, nrhs, _dptr(x), _dptr(pp), _dptr(qm), precision))
        return pp, qm

    def reflect(self, p_plus, q_minus):
        pp = _c128(p_plus).reshape(-1, self.ns)
        qm = _c128(q_minus).reshape(-1, self.ns)
        sp, sm = np.zeros_like(pp), np.zeros_like(qm)
        self._check(self.lib.lsms_reflect(self.h, pp.shape[0], _dptr(pp), _dptr(qm), _dptr(sp), _dptr(sm)))
        return sp, sm

    def disaggregate(self, s_plus, s_minus, precision=LSMS_FP64):
        sp = _c128(s_plus).reshape(-1, self.ns)
        sm = _c128(s_minus).reshape(-1, self.ns)
        a = np.zeros((sp.shape[0], self.n, self.P), dtype=np.complex128)
        self._check(self.lib.lsms_disaggregate(self.h, sp.shape[0], _dptr(sp), _dptr(sm), _dptr(a), precision))
        return a

    def incident(self, sources):
        s = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 2)
        a = np.zeros((s.shape[0], self.n, self.P), dtype=np.complex128)
        self._check(self.lib.lsms_incident(self.h, s.shape[0], _dptr(s), _dptr(a)))
        return a

    def set_timing(self, enable=True):
        self._check(self.lib.lsms_set_timing(self.h, 1 if enable else 0))

    def last_timing(self):
        """(ms of the translation, ms of the reflected coupling, kernels launched) of the last apply."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        self._check(self.lib.lsms_last_timing(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
        return a.value, b.value, n.value

    # -- solve and fields --------------------------------------------------------------------------
    def solve(self, sources, tol=1e-10, maxiter=500, x0=None, history=0, raise_on_error=True):
        s = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 2)
        if getattr(self, "layout_counts", None) is not None:
            beta = np.zeros((self.n, self.P), dtype=np.complex128)    # one array per layout, joined
        else:
            beta = np.zeros((s.shape[0], self.n, self.P), dtype=np.complex128)
        info = SolveInfo()
        hist = np.zeros(max(history, 1))
        info.history = hist.ctypes.data_as(_D)
        info.history_cap = history
        x0a = None if x0 is None else _c128(x0, beta.shape)
        if getattr(self, "layout_counts", None) is not None and x0 is not None:
            x0a = _c128(x0, beta.shape)
        rc = self.lib.lsms_solve(self.h, s.shape[0], _dptr(s), tol, maxiter, _dptr(x0a), _dptr(beta),
                                 ctypes.byref(info))
        if raise_on_error:
            self._check(rc)
        out = dict(status=rc, iters=info.iters, outer_iters=info.outer_iters, rel_res=info.rel_res,
                   rel_res_fp64=info.rel_res_fp64, history=hist[:info.n_history].copy())
        return beta, out

    def eval_field(self, targets, src_index=0, which=FIELD_TOTAL):
        t = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 2)
        u = np.zeros(t.shape[0], dtype=np.complex128)
        self._check(self.lib.lsms_eval_field(self.h, src_index, t.shape[0], _dptr(t), which, _dptr(u)))
        return u


def build_contour(n_nodes, k1, k2, k3, b=0.0, t_max=0.0, panel_order=0, panel_rule=0):
    """Host-only: the library's contour nodes and weights (no GPU needed)."""
    lib = load()
    lam = np.zeros(n_nodes, dtype=np.complex128)
    wt = np.zeros(n_nodes, dtype=np.complex128)
    c = Contour(n_nodes, b, t_max, panel_order, panel_rule)
    rc = lib.lsms_build_contour(ctypes.byref(c), k1, k2, k3, _dptr(lam), _dptr(wt))
    if rc != 0:
        raise LsmsError(rc, lib.lsms_last_error(None).decode())
    return lam, wt


def build_contour_stack(n_nodes, ks, b=0.0, t_max=0.0, panel_order=0, panel_rule=0):
    """Host-only: the library's contour for a stack of layers with wavenumbers ks (top to bottom)."""
    lib = load()
    k = np.ascontiguousarray(np.real(np.asarray(ks)), dtype=np.float64)
    lam = np.zeros(n_nodes, dtype=np.complex128)
    wt = np.zeros(n_nodes, dtype=np.complex128)
    c = Contour(n_nodes, b, t_max, panel_order, panel_rule)
    rc = lib.lsms_build_contour_stack(ctypes.byref(c), int(k.size), _dptr(k), _dptr(lam), _dptr(wt))
    if rc != 0:
        raise LsmsError(rc, lib.lsms_last_error(None).decode())
    return lam, wt


def layer_response(ks, thicknesses, particle_layer, lam) -> np.ndarray:
    """Host-only: (n, 4, 3) complex, rows sigma_1, s_m^+, s_m^-, sigma_L for unit I, P, Q."""
    lib = load()
    k = np.ascontiguousarray(np.asarray(ks, dtype=np.complex128))
    ds = np.ascontiguousarray(thicknesses, dtype=np.float64)
    lm = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128).ravel())
    out = np.zeros((lm.size, 4, 3), dtype=np.complex128)
    rc = lib.lsms_layer_response(int(k.size), _dptr(k), _dptr(ds), int(particle_layer), int(lm.size), _dptr(lm),
                                 _dptr(out))
    if rc != 0:
        raise LsmsError(rc, lib.lsms_last_error(None).decode())
    return out


def scattering_diagonal(p, k2, kp, radius):
    """Host-only: the library's disc scattering matrix diagonal S_n, n = -p..p; a complex kp (an
    absorbing disc) goes to lsms_scattering_diagonal_c."""
    lib = load()
    s = np.zeros(2 * p + 1, dtype=np.complex128)
    if np.iscomplexobj(kp):
        kc = complex(kp)
        rc = lib.lsms_scattering_diagonal_c(int(p), float(k2), kc.real, kc.imag, float(radius), _dptr(s))
    else:
        rc = lib.lsms_scattering_diagonal(p, k2, kp, radius, _dptr(s))
    if rc != 0:
        raise LsmsError(rc, lib.lsms_last_error(None).decode())
    return s


def check_geometry(d, radius, centres) -> int:
    """Host-only: LSMS_OK (0) or a negative status for a disc layout."""
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 2)
    return load().lsms_check_geometry(d, radius, c.shape[0], _dptr(c))


def translate_mixed_noalloc(centres, beta, alpha, k2, p, stream=None):
    """FP32 translation with no device allocation (lsms_translate_mixed_noalloc).

    centres: CUDA float64 tensor (n, 2); beta, alpha: CUDA complex128 tensors (nrhs, n, 2p+1).
    Asynchronous on `stream` (default: torch's current stream)."""
    import torch
    lib = load()
    p = int(p)
    dev = torch.cuda.current_device()
    for name, t, dt in (("centres", centres, torch.float64), ("beta", beta, torch.complex128),
                        ("alpha", alpha, torch.complex128)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"translate_mixed_noalloc: {name} must be a torch tensor")
        if not t.is_cuda or t.device.index != dev:
            raise ValueError(f"translate_mixed_noalloc: {name} must be on the current CUDA device (cuda:{dev}), "
                             f"got {t.device}")
        if t.dtype != dt:
            raise ValueError(f"translate_mixed_noalloc: {name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"translate_mixed_noalloc: {name} must be contiguous")
    if centres.dim() != 2 or centres.shape[1] != 2:
        raise ValueError(f"translate_mixed_noalloc: centres must have shape (n, 2), got {tuple(centres.shape)}")
    n = centres.shape[0]
    P = 2 * p + 1
    if p < 0:
        raise ValueError("translate_mixed_noalloc: p must be >= 0")
    if n == 0:
        nrhs = 0
        if beta.numel() != 0:
            raise ValueError("translate_mixed_noalloc: beta must be empty when there are no discs")
    elif beta.numel() % (n * P) != 0:
        raise ValueError(f"translate_mixed_noalloc: beta ({beta.numel()} elements) is not nrhs x {n} x {P}")
    else:
        nrhs = beta.numel() // (n * P)
    if alpha.shape != beta.shape:
        raise ValueError(f"translate_mixed_noalloc: alpha {tuple(alpha.shape)} and beta {tuple(beta.shape)} differ")
    if stream is None:
        stream = torch.cuda.current_stream()
    rc = lib.lsms_translate_mixed_noalloc(n, p, k2, nrhs, ctypes.c_void_p(centres.data_ptr()),
                                          ctypes.c_void_p(beta.data_ptr()),
                                          ctypes.c_void_p(alpha.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream))
    if rc != 0:
        raise LsmsError(rc, lib.lsms_last_error(None).decode())


def inclusion_scattering_matrix(p, k2, kp, radius, curve) -> np.ndarray:
    """lsms_inclusion_scattering_matrix: curve = (x, x', x'') as three (n_pts, 2) arrays; a complex
    kp (an absorbing inclusion) goes to lsms_inclusion_scattering_matrix_c."""
    lib = load()
    x, dx, ddx = (np.asarray(a, dtype=np.float64).reshape(-1, 2) for a in curve)
    c = np.ascontiguousarray(np.concatenate([x, dx, ddx], axis=1))
    s = np.zeros((2 * p + 1, 2 * p + 1), dtype=np.complex128)
    if np.iscomplexobj(kp):
        kc = complex(kp)
        rc = lib.lsms_inclusion_scattering_matrix_c(int(p), float(k2), kc.real, kc.imag, float(radius), c.shape[0],
                                                    _dptr(c), _dptr(s))
    else:
        rc = lib.lsms_inclusion_scattering_matrix(int(p), float(k2), float(kp), float(radius), c.shape[0],
                                                  _dptr(c), _dptr(s))
    if rc != 0:
        raise LsmsError(rc, lib.lsms_last_error(None).decode())
    return s


def pec_scattering_diagonal(p, k2, radius) -> np.ndarray:
    """lsms_pec_scattering_diagonal: S_n of a perfectly conducting disc, n = -p..p."""
    lib = load()
    s = np.zeros(2 * p + 1, dtype=np.complex128)
    rc = lib.lsms_pec_scattering_diagonal(int(p), float(k2), float(radius), _dptr(s))
    if rc != 0:
        raise LsmsError(rc, lib.lsms_last_error(None).decode())
    return s


def context_for(workload, precision=LSMS_FP64) -> Context:
    """A context for one of paper_1407_3868_gb300.inputs.WORKLOADS (medium, p, contour)."""
    m = workload.medium
    return Context(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"], workload.p,
                   workload.n_nodes, b=workload.b, t_max=workload.t_max, panel_order=16,
                   precision=precision)
