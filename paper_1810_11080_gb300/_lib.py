"""ctypes binding of libsnsweep.so (include/snsweep.h): argument marshalling only.

Every function keeps the C name.  Array arguments may be numpy arrays (host memory) or torch
tensors (host or CUDA); they are passed as raw pointers after a dtype/contiguity check.
The library must have been built (paper_1810_11080_gb300.build.build()); importing this
module without it raises immediately -- there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsnsweep.so")

SN_OK, SN_EINVAL, SN_ENOMEM, SN_ECUDA, SN_ETIMEOUT, SN_ENOTCONVERGED, SN_EMESH, SN_ESTATE = range(8)
SN_WEIGHT_UNITY, SN_WEIGHT_FACE, SN_WEIGHT_SIGINVFACE = 0, 1, 2
SN_PREC_FP64, SN_PREC_MIXED, SN_PREC_MIXED_DS, SN_PREC_FP64_INV, SN_PREC_DS_INV = 0, 1, 2, 3, 4
SN_LAUNCH_LEVELS, SN_LAUNCH_DATAFLOW = 0, 1
WEIGHTING = {"unity": 0, "face": 1, "siginvface": 2}

EXPORTED = ["sn_create", "sn_destroy", "sn_last_error", "sn_set_mesh", "sn_set_discretization",
            "sn_set_quadrature", "sn_set_materials", "sn_num_boundary_faces", "sn_build_graph",
            "sn_get_graph", "sn_sweep", "sn_moment", "sn_source_iterate", "sn_si_begin", "sn_si_step",
            "sn_si_result", "sn_kernel_launches", "sn_moment_noalloc", "sn_set_launch", "sn_autotune",
            "sn_batch_create", "sn_batch_destroy", "sn_batch_last_error", "sn_batch_updates_per_sweep",
            "sn_batch_set_launch", "sn_batch_tune", "sn_batch_si_begin", "sn_batch_si_step",
            "sn_batch_source_iterate", "sn_mlp_create", "sn_mlp_destroy", "sn_mlp_num_params", "sn_mlp_params",
            "sn_mlp_forward", "sn_mlp_grad", "sn_mlp_train", "sn_predictor_features", "sn_predictor_init_targets",
            "sn_predictor_corr_data", "sn_source_iterate_learned", "sn_predictor_initial_phi",
            "sn_quadrature_level_symmetric", "sn_set_spin_limit", "sn_set_dsa", "sn_dsa_correction",
            "sn_dsa_last_iters", "sn_prepare_inverse", "sn_release_inverse", "sn_num_volume_points",
            "sn_volume_points", "sn_l2_error", "sn_set_mesh_simplex"]


class sn_graph_stats(ctypes.Structure):
    _fields_ = [("n_arcs", ctypes.c_int64), ("n_removed", ctypes.c_int64), ("n_scc", ctypes.c_int64),
                ("max_scc", ctypes.c_int32), ("max_level", ctypes.c_int32), ("n_mixed_faces", ctypes.c_int64),
                ("ms_geometry", ctypes.c_double), ("ms_weights", ctypes.c_double), ("ms_fas", ctypes.c_double),
                ("ms_levels", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sn_si_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("residual", ctypes.c_double),
                ("ms_total", ctypes.c_double)]


SN_FEATURES = 16


class sn_predictor_cfg(ctypes.Structure):
    _fields_ = [("init_mean", ctypes.c_float * SN_FEATURES), ("init_istd", ctypes.c_float * SN_FEATURES),
                ("corr_mean", ctypes.c_float * (SN_FEATURES + 2)), ("corr_istd", ctypes.c_float * (SN_FEATURES + 2)),
                ("corr_start", ctypes.c_int32), ("corr_every", ctypes.c_int32)]


class SnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"snsweep status {status}: {msg}")
        self.status = status


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1810_11080_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "sn_create": (I, [ctypes.POINTER(P), I, P]),
        "sn_destroy": (None, [P]),
        "sn_last_error": (ctypes.c_char_p, [P]),
        "sn_set_mesh": (I, [P, I, I64, I, P, P, P, P]),
        "sn_set_discretization": (I, [P, I, I]),
        "sn_set_quadrature": (I, [P, I, P, P]),
        "sn_set_materials": (I, [P, P, P, P, P, P]),
        "sn_num_boundary_faces": (I64, [P]),
        "sn_build_graph": (I, [P, I, I, ctypes.POINTER(sn_graph_stats)]),
        "sn_get_graph": (I, [P, ctypes.POINTER(I64), P, I64, P]),
        "sn_sweep": (I, [P, P, P, P, I]),
        "sn_moment": (I, [P, P, P, P, ctypes.POINTER(D)]),
        "sn_source_iterate": (I, [P, D, I, I, P, P, P, ctypes.POINTER(sn_si_stats), P, I]),
        "sn_si_begin": (I, [P, P]),
        "sn_si_step": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_float)]),
        "sn_si_result": (I, [P, P, P]),
        "sn_kernel_launches": (I64, [P]),
        "sn_set_launch": (I, [P, I, I]),
        "sn_autotune": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "sn_batch_create": (I, [ctypes.POINTER(P), I, P, P]),
        "sn_batch_destroy": (None, [P]),
        "sn_batch_last_error": (ctypes.c_char_p, [P]),
        "sn_batch_updates_per_sweep": (I64, [P]),
        "sn_batch_set_launch": (I, [P, I, I]),
        "sn_batch_tune": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "sn_batch_si_begin": (I, [P, P]),
        "sn_predictor_initial_phi": (I, [P, P, ctypes.POINTER(sn_predictor_cfg), P]),
        "sn_batch_si_step": (I, [P, I, P, ctypes.POINTER(ctypes.c_float)]),
        "sn_batch_source_iterate": (I, [P, D, I, I, P, P, ctypes.POINTER(D)]),
        "sn_mlp_create": (I, [ctypes.POINTER(P), I, P, I, I, ctypes.c_uint64]),
        "sn_mlp_destroy": (None, [P]),
        "sn_mlp_num_params": (I64, [P]),
        "sn_mlp_params": (I, [P, P, P]),
        "sn_mlp_forward": (I, [P, I64, P, P]),
        "sn_mlp_grad": (I, [P, I64, P, P, ctypes.POINTER(ctypes.c_float), P]),
        "sn_mlp_train": (I, [P, I64, P, P, I, I, ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)]),
        "sn_predictor_features": (I, [P, P, P]),
        "sn_predictor_init_targets": (I, [P, P, P]),
        "sn_predictor_corr_data": (I, [P, P, P, P, P, P, P]),
        "sn_source_iterate_learned": (I, [P, D, I, I, P, P, ctypes.POINTER(sn_predictor_cfg), P,
                                          ctypes.POINTER(sn_si_stats), ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
        "sn_moment_noalloc": (I, [I, P, I, I64, I, P, P, P, P, ctypes.POINTER(D)]),
        "sn_quadrature_level_symmetric": (I, [I, I, ctypes.POINTER(I), P, P]),
        "sn_set_spin_limit": (I, [P, I64]),
        "sn_set_dsa": (I, [P, I, D, I]),
        "sn_dsa_correction": (I, [P, P, P, P, ctypes.POINTER(I)]),
        "sn_dsa_last_iters": (ctypes.c_int32, [P]),
        "sn_prepare_inverse": (I, [P, I, ctypes.POINTER(ctypes.c_float)]),
        "sn_release_inverse": (I, [P]),
        "sn_num_volume_points": (ctypes.c_int32, [P]),
        "sn_volume_points": (I, [P, P]),
        "sn_l2_error": (I, [P, P, P, ctypes.POINTER(D)]),
        "sn_set_mesh_simplex": (I, [P, I, I64, I, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _ptr(a, dtype, name):
    """Raw pointer of a numpy array or torch tensor of the given numpy dtype (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"{name}: expected C-contiguous {np.dtype(dtype).name} array")
        return a.ctypes.data
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        tmap = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32, np.float32: torch.float32}
        if a.dtype != tmap[np.dtype(dtype).type] or not a.is_contiguous():
            raise TypeError(f"{name}: expected contiguous {tmap[np.dtype(dtype).type]} tensor")
        return a.data_ptr()
    raise TypeError(f"{name}: expected numpy array or torch tensor")


def sn_moment_noalloc(device, stream, w, psi, phi_prev, phi_out):
    """Context-free scalar-flux moment for callers that cannot allocate device memory (see
    include/snsweep.h).  All arrays are CUDA tensors; psi [n_dir][n_elem][n_dofs].  Returns the
    relative scalar-flux change."""
    n_dir, n_elem, n_dofs = psi.shape
    r = ctypes.c_double()
    st = lib().sn_moment_noalloc(int(device), stream, int(n_dir), int(n_elem), int(n_dofs), _ptr(w, np.float64, "w"),
                                 _ptr(psi, np.float64, "psi"), _ptr(phi_prev, np.float64, "phi_prev"),
                                 _ptr(phi_out, np.float64, "phi_out"), ctypes.byref(r))
    if st != SN_OK:
        raise SnError(st, "sn_moment_noalloc failed (device pointers only; n_elem*n_dofs <= 4194304)")
    return r.value


def sn_quadrature_level_symmetric(N, dim):
    """Level-symmetric S_N set from the library (host arrays): returns (omega [M][3], w [M])."""
    n = ctypes.c_int()
    st = lib().sn_quadrature_level_symmetric(int(N), int(dim), ctypes.byref(n), None, None)
    if st != SN_OK:
        raise SnError(st, f"sn_quadrature_level_symmetric(N={N}, dim={dim}) failed")
    omega = np.zeros((n.value, 3))
    w = np.zeros(n.value)
    st = lib().sn_quadrature_level_symmetric(int(N), int(dim), ctypes.byref(n), omega.ctypes.data, w.ctypes.data)
    if st != SN_OK:
        raise SnError(st, f"sn_quadrature_level_symmetric(N={N}, dim={dim}) failed")
    return omega, w


class Context:
    """Owns one sn_ctx.  Methods map one to one onto the C functions."""

    def __init__(self, device=0, stream=None):
        self._lib = lib()
        self._c = ctypes.c_void_p()
        st = self._lib.sn_create(ctypes.byref(self._c), int(device), stream)
        if st != SN_OK:
            raise SnError(st, "sn_create failed")

    def _check(self, st):
        if st != SN_OK:
            raise SnError(st, self._lib.sn_last_error(self._c).decode())
        return st

    def close(self):
        if self._c:
            self._lib.sn_destroy(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sn_set_mesh_simplex(self, dim, n_elem, r, ctrl, face_nbr, nbr_face, orient):
        self._n_elem = int(n_elem)
        self._dim = int(dim)
        return self._check(self._lib.sn_set_mesh_simplex(self._c, dim, n_elem, r, _ptr(ctrl, np.float64, "ctrl"),
                                                         _ptr(face_nbr, np.int64, "face_nbr"),
                                                         _ptr(nbr_face, np.int32, "nbr_face"),
                                                         _ptr(orient, np.int32, "orient")))

    def sn_set_mesh(self, dim, n_elem, r, ctrl, face_nbr, nbr_face, orient):
        self._n_elem = int(n_elem)
        self._dim = int(dim)
        return self._check(self._lib.sn_set_mesh(self._c, dim, n_elem, r, _ptr(ctrl, np.float64, "ctrl"),
                                                 _ptr(face_nbr, np.int64, "face_nbr"),
                                                 _ptr(nbr_face, np.int32, "nbr_face"),
                                                 _ptr(orient, np.int32, "orient")))

    def sn_set_discretization(self, p, face_subdiv=2):
        self._p = int(p)
        return self._check(self._lib.sn_set_discretization(self._c, p, face_subdiv))

    def sn_set_quadrature(self, omega, w):
        return self._check(self._lib.sn_set_quadrature(self._c, len(w), _ptr(omega, np.float64, "omega"),
                                                       _ptr(w, np.float64, "w")))

    def sn_set_materials(self, sigma_t, sigma_s, q=None, q_dir=None, psi_inc=None):
        return self._check(self._lib.sn_set_materials(self._c, _ptr(sigma_t, np.float64, "sigma_t"),
                                                      _ptr(sigma_s, np.float64, "sigma_s"),
                                                      _ptr(q, np.float64, "q"), _ptr(q_dir, np.float64, "q_dir"),
                                                      _ptr(psi_inc, np.float64, "psi_inc")))

    def sn_num_boundary_faces(self):
        return self._lib.sn_num_boundary_faces(self._c)

    def sn_build_graph(self, weighting="face", exact_max=10):
        st = sn_graph_stats()
        w = WEIGHTING[weighting] if isinstance(weighting, str) else int(weighting)
        self._check(self._lib.sn_build_graph(self._c, w, exact_max, ctypes.byref(st)))
        return st.as_dict()

    def sn_get_graph(self, n_dir, n_elem):
        n = ctypes.c_int64()
        self._check(self._lib.sn_get_graph(self._c, ctypes.byref(n), None, 0, None))
        removed = np.zeros((max(1, n.value), 3), dtype=np.int32)
        levels = np.zeros((n_dir, n_elem), dtype=np.int32)
        self._check(self._lib.sn_get_graph(self._c, ctypes.byref(n), removed.ctypes.data, n.value,
                                           levels.ctypes.data))
        return removed[:n.value].astype(np.int64), levels

    def sn_sweep(self, phi_in, psi_old, psi_new, precision=SN_PREC_FP64):
        return self._check(self._lib.sn_sweep(self._c, _ptr(phi_in, np.float64, "phi_in"),
                                              _ptr(psi_old, np.float64, "psi_old"),
                                              _ptr(psi_new, np.float64, "psi_new"), precision))

    def sn_moment(self, psi, phi_prev, phi_out):
        r = ctypes.c_double()
        self._check(self._lib.sn_moment(self._c, _ptr(psi, np.float64, "psi"),
                                        _ptr(phi_prev, np.float64, "phi_prev"),
                                        _ptr(phi_out, np.float64, "phi_out"), ctypes.byref(r)))
        return r.value

    def sn_source_iterate(self, tol, max_iter, precision=SN_PREC_FP64, phi0=None, phi_out=None, psi_out=None,
                          history_cap=0):
        st = sn_si_stats()
        hist = np.zeros(max(1, history_cap))
        s = self._lib.sn_source_iterate(self._c, tol, max_iter, precision, _ptr(phi0, np.float64, "phi0"),
                                        _ptr(phi_out, np.float64, "phi_out"), _ptr(psi_out, np.float64, "psi_out"),
                                        ctypes.byref(st), hist.ctypes.data if history_cap else None, history_cap)
        if s not in (SN_OK, SN_ENOTCONVERGED):
            self._check(s)
        return dict(status=s, iters=st.iters, converged=bool(st.converged), residual=st.residual,
                    ms_total=st.ms_total, history=hist[:min(st.iters, history_cap)].copy())

    def sn_set_launch(self, mode, blocks_per_sm=0):
        return self._check(self._lib.sn_set_launch(self._c, int(mode), int(blocks_per_sm)))

    def sn_set_dsa(self, enable=True, rtol=1e-4, max_iter=500):
        en = int(enable) if not isinstance(enable, bool) else (1 if enable else 0)
        return self._check(self._lib.sn_set_dsa(self._c, en, float(rtol), int(max_iter)))

    def sn_dsa_correction(self, phi_half, phi_prev, phi_out):
        it = ctypes.c_int()
        self._check(self._lib.sn_dsa_correction(self._c, _ptr(phi_half, np.float64, "phi_half"),
                                                _ptr(phi_prev, np.float64, "phi_prev"),
                                                _ptr(phi_out, np.float64, "phi_out"), ctypes.byref(it)))
        return it.value

    def sn_dsa_last_iters(self):
        return self._lib.sn_dsa_last_iters(self._c)

    def sn_prepare_inverse(self, precision=SN_PREC_FP64_INV):
        """Forms the stored local inverses and face blocks of a stored-inverse form; returns device ms."""
        ms = ctypes.c_float()
        self._check(self._lib.sn_prepare_inverse(self._c, int(precision), ctypes.byref(ms)))
        return ms.value

    def sn_release_inverse(self):
        return self._check(self._lib.sn_release_inverse(self._c))

    def sn_volume_points(self):
        """[n_elem][Q][dim] physical positions of the volume quadrature points."""
        Q = self._lib.sn_num_volume_points(self._c)
        out = np.zeros((self._n_elem, Q, self._dim))
        self._check(self._lib.sn_volume_points(self._c, _ptr(out, np.float64, "xq")))
        return out

    def sn_l2_error(self, phi, exact_q):
        err = ctypes.c_double()
        self._check(self._lib.sn_l2_error(self._c, _ptr(phi, np.float64, "phi"), _ptr(exact_q, np.float64, "exact_q"),
                                          ctypes.byref(err)))
        return err.value

    def sn_set_spin_limit(self, polls):
        return self._check(self._lib.sn_set_spin_limit(self._c, int(polls)))

    def sn_autotune(self, precision=SN_PREC_MIXED_DS):
        m, b = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.sn_autotune(self._c, int(precision), ctypes.byref(m), ctypes.byref(b)))
        return m.value, b.value

    def sn_si_begin(self, phi0=None):
        return self._check(self._lib.sn_si_begin(self._c, _ptr(phi0, np.float64, "phi0")))

    def sn_si_step(self, precision=SN_PREC_FP64, time_sweep=False):
        """Returns (residual, sweep milliseconds or None)."""
        r = ctypes.c_double()
        ms = ctypes.c_float()
        self._check(self._lib.sn_si_step(self._c, precision, ctypes.byref(r), ctypes.byref(ms) if time_sweep else None))
        return r.value, (ms.value if time_sweep else None)

    def sn_si_result(self, phi_out=None, psi_out=None):
        return self._check(self._lib.sn_si_result(self._c, _ptr(phi_out, np.float64, "phi_out"),
                                                  _ptr(psi_out, np.float64, "psi_out")))

    def sn_predictor_features(self):
        E = self._n_elem
        feat = np.zeros((E, SN_FEATURES), dtype=np.float32)
        ref = np.zeros(E)
        self._check(self._lib.sn_predictor_features(self._c, feat.ctypes.data, ref.ctypes.data))
        return feat, ref

    def sn_predictor_init_targets(self, phi):
        t = np.zeros(phi.shape, dtype=np.float32)
        self._check(self._lib.sn_predictor_init_targets(self._c, _ptr(phi, np.float64, "phi"), t.ctypes.data))
        return t

    def sn_predictor_corr_data(self, phi_a, phi_b, phi_c, phi_inf=None):
        E = phi_a.shape[0]
        x = np.zeros((E, SN_FEATURES + 2), dtype=np.float32)
        t = np.zeros(E, dtype=np.float32) if phi_inf is not None else None
        self._check(self._lib.sn_predictor_corr_data(self._c, _ptr(phi_a, np.float64, "phi_a"),
                                                     _ptr(phi_b, np.float64, "phi_b"), _ptr(phi_c, np.float64, "phi_c"),
                                                     _ptr(phi_inf, np.float64, "phi_inf"), x.ctypes.data,
                                                     None if t is None else t.ctypes.data))
        return x, t

    def sn_predictor_initial_phi(self, init_model, cfg):
        phi = np.zeros((self._n_elem, self._N))
        self._check(self._lib.sn_predictor_initial_phi(self._c, init_model._m, ctypes.byref(cfg), phi.ctypes.data))
        return phi

    def sn_source_iterate_learned(self, tol, max_iter, precision, init_model, corr_model, cfg, phi_out=None):
        st = sn_si_stats()
        acc, rej = ctypes.c_int32(), ctypes.c_int32()
        s = self._lib.sn_source_iterate_learned(self._c, float(tol), int(max_iter), int(precision),
                                                None if init_model is None else init_model._m,
                                                None if corr_model is None else corr_model._m, ctypes.byref(cfg),
                                                _ptr(phi_out, np.float64, "phi_out"), ctypes.byref(st),
                                                ctypes.byref(acc), ctypes.byref(rej))
        if s not in (SN_OK, SN_ENOTCONVERGED):
            self._check(s)
        return dict(status=s, iters=st.iters, converged=bool(st.converged), residual=st.residual,
                    ms_total=st.ms_total, accepted=acc.value, rejected=rej.value)

    def sn_kernel_launches(self):
        return self._lib.sn_kernel_launches(self._c)


class Batch:
    """Owns one sn_batch over a list of Contexts (which must outlive it)."""

    def __init__(self, contexts, stream=None):
        self._lib = lib()
        self._ctxs = list(contexts)
        arr = (ctypes.c_void_p * len(self._ctxs))(*[c._c.value for c in self._ctxs])
        self._b = ctypes.c_void_p()
        st = self._lib.sn_batch_create(ctypes.byref(self._b), len(self._ctxs), arr, stream)
        if st != SN_OK:
            raise SnError(st, "sn_batch_create failed (contexts must share device and dimension and have graphs)")

    def _check(self, st):
        if st != SN_OK:
            raise SnError(st, self._lib.sn_batch_last_error(self._b).decode())
        return st

    def close(self):
        if self._b:
            self._lib.sn_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sn_batch_updates_per_sweep(self):
        return self._lib.sn_batch_updates_per_sweep(self._b)

    def sn_batch_set_launch(self, mode, blocks_per_sm=0):
        return self._check(self._lib.sn_batch_set_launch(self._b, int(mode), int(blocks_per_sm)))

    def sn_batch_tune(self, precision=SN_PREC_MIXED_DS):
        m, b = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.sn_batch_tune(self._b, int(precision), ctypes.byref(m), ctypes.byref(b)))
        return m.value, b.value

    def sn_batch_si_begin(self, phi0=None):
        """phi0: None or a list of per-problem arrays (or None entries)."""
        if phi0 is None:
            return self._check(self._lib.sn_batch_si_begin(self._b, None))
        keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in phi0]
        arr = (ctypes.c_void_p * len(keep))(*[None if a is None else a.ctypes.data for a in keep])
        return self._check(self._lib.sn_batch_si_begin(self._b, arr))

    def sn_batch_si_step(self, precision=SN_PREC_MIXED_DS, time_sweep=False):
        res = np.zeros(len(self._ctxs))
        ms = ctypes.c_float()
        self._check(self._lib.sn_batch_si_step(self._b, int(precision), res.ctypes.data,
                                               ctypes.byref(ms) if time_sweep else None))
        return res, (ms.value if time_sweep else None)

    def sn_batch_source_iterate(self, tol, max_iter, precision=SN_PREC_MIXED_DS):
        its = np.zeros(len(self._ctxs), dtype=np.int32)
        res = np.zeros(len(self._ctxs))
        ms = ctypes.c_double()
        st = self._lib.sn_batch_source_iterate(self._b, float(tol), int(max_iter), int(precision), its.ctypes.data,
                                               res.ctypes.data, ctypes.byref(ms))
        if st not in (SN_OK, SN_ENOTCONVERGED):
            self._check(st)
        return dict(status=st, iters=its, residuals=res, ms_total=ms.value)


class MLP:
    """Owns one sn_mlp (3 layers, width 64, BF16 weights)."""

    def __init__(self, n_in, n_out, seed=0, device=0, stream=None):
        self._lib = lib()
        self._m = ctypes.c_void_p()
        self.n_in, self.n_out = n_in, n_out
        st = self._lib.sn_mlp_create(ctypes.byref(self._m), int(device), stream, int(n_in), int(n_out), int(seed))
        if st != SN_OK:
            raise SnError(st, "sn_mlp_create failed")

    def _check(self, st, what="sn_mlp"):
        if st != SN_OK:
            raise SnError(st, f"{what} failed")
        return st

    def close(self):
        if self._m:
            self._lib.sn_mlp_destroy(self._m)
            self._m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sn_mlp_num_params(self):
        return self._lib.sn_mlp_num_params(self._m)

    def get_params(self):
        p = np.zeros(self.sn_mlp_num_params(), dtype=np.float32)
        self._check(self._lib.sn_mlp_params(self._m, p.ctypes.data, None))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self._lib.sn_mlp_params(self._m, None, p.ctypes.data))

    def sn_mlp_forward(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros((x.shape[0], self.n_out), dtype=np.float32)
        self._check(self._lib.sn_mlp_forward(self._m, x.shape[0], x.ctypes.data, y.ctypes.data))
        return y

    def sn_mlp_grad(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(self.sn_mlp_num_params(), dtype=np.float32)
        L = ctypes.c_float()
        self._check(self._lib.sn_mlp_grad(self._m, x.shape[0], x.ctypes.data, t.ctypes.data, ctypes.byref(L),
                                          g.ctypes.data))
        return L.value, g

    def sn_mlp_train(self, x, t, epochs, batch_rows=4096, lr=1e-3, seed=0):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        L = ctypes.c_float()
        self._check(self._lib.sn_mlp_train(self._m, x.shape[0], x.ctypes.data, t.ctypes.data, int(epochs),
                                           int(batch_rows), float(lr), int(seed), ctypes.byref(L)))
        return L.value
