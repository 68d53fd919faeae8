"""Python binding of the GB300 PIC library (libpic.so, C ABI in include/pic.h).

Argument marshalling only: every step of the PIC loop runs in the library's
CUDA kernels. PyTorch supplies device memory and the CUDA stream. If the
shared library has not been built the import of any binding call raises,
there is no CPU fallback.

Module-level functions carry the C names (``pic_create``, ``pic_init``,
``pic_deposit``, ``poisson_solve``, ``poisson_solve_ex``, ``pic_gather_push``,
``pic_sync_velocity``, ``pic_field_energy``, ``pic_get_particles``,
``pic_apply_laplacian``, ``pic_profile_enable``, ``pic_profile_read``,
``pic_destroy``); ``Context`` bundles them, and calls the other entry points
(the spectral solve ``pic_fft_solve``, the particle-in-Fourier
``pic_pif_field`` and ``pic_pif_push``, ``pic_gather_push_field``,
``pic_sync_velocity_field``, ``pic_field_energy_E``, the learned
preconditioner's and the V-cycle's) as methods.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

PIC_OK = 0
PIC_EINVAL = -1
PIC_ENOMEM = -2
PIC_ECUDA = -3
PIC_ENOCONV = -4
PIC_EBREAKDOWN = -5
PIC_ETIMEOUT = -6
PIC_ESTATE = -7

PREC_FP64 = 0
PREC_MIXED = 1
PC_JACOBI = 0
PC_CNN = 1
PC_MG = 2
PC_MG_CNN = 3
PC_SSOR = 4
CNN_APPLY_TC = 0
CNN_APPLY_FP32 = 1
CNN_APPLY_LAYERS = 2
CNN_APPLY_TC_FUSED = 3
CNN_APPLY_TC8 = 4
CNN_WEIGHTS = 14688
CNN_TRAIN_BF16 = 0
CNN_TRAIN_FP32 = 1


class PicError(RuntimeError):
    def __init__(self, code, what):
        detail = ""
        if code == PIC_ECUDA:
            try:
                detail = f" [{lib().pic_cuda_error().decode()}]"
            except ImportError:
                pass
        super().__init__(f"{what}: {strerror(code)} ({code}){detail}")
        self.code = code


class pic_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("ppc", ctypes.c_int), ("alpha", ctypes.c_double), ("k", ctypes.c_double),
                ("vth", ctypes.c_double), ("init_mode", ctypes.c_int)]


class pic_solve_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("precond", ctypes.c_int), ("reliable_delta", ctypes.c_double),
                ("check_every", ctypes.c_int), ("refine_max", ctypes.c_int)]


class pic_profile_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("phase_calls", ctypes.c_int * 4), ("phase_ms", ctypes.c_double * 4),
                ("ker_samples", ctypes.c_int * 14), ("ker_ms", ctypes.c_double * 14),
                ("ker_precision", ctypes.c_int * 14)]

    def as_dict(self):
        phases = ("deposit", "solve", "push", "energy")
        kers = ("pap", "update", "precond", "dot", "mg_pre", "mg_resid", "mg_restrict", "mg_prolong_smooth",
                "mg_smooth", "scatter", "deposit", "push", "pif_spread", "pif_gather")
        return {
            "launches": int(self.launches),
            "phase_calls": {p: self.phase_calls[i] for i, p in enumerate(phases)},
            "phase_ms": {p: self.phase_ms[i] for i, p in enumerate(phases)},
            "ker_samples": {k: self.ker_samples[i] for i, k in enumerate(kers)},
            "ker_ms": {k: self.ker_ms[i] for i, k in enumerate(kers)},
            "ker_precision": {k: self.ker_precision[i] for i, k in enumerate(kers)},
        }


TRAIN_PRECONDITIONER = 0
TRAIN_SMOOTHER = 1


class pic_train_opts(ctypes.Structure):
    _fields_ = [("target", ctypes.c_int), ("grid", ctypes.c_int), ("sets", ctypes.c_int), ("steps", ctypes.c_int),
                ("batch", ctypes.c_int), ("crop", ctypes.c_int), ("lr", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("validate_every", ctypes.c_int), ("val_grid", ctypes.c_int), ("val_seed", ctypes.c_uint64),
                ("resume", ctypes.c_int), ("restarts", ctypes.c_int)]


class pic_train_info(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("adam_steps", ctypes.c_int), ("best_step", ctypes.c_int),
                ("best_iters", ctypes.c_int), ("best_restart", ctypes.c_int), ("loss_first", ctypes.c_double),
                ("loss_last", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pic_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("fallbacks", ctypes.c_int),
                ("converged", ctypes.c_int), ("rel_res", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("t_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

# symbol -> (restype, argtypes)
_SIGS = {
    "pic_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pic_cuda_error": (ctypes.c_char_p, []),
    "pic_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "pic_destroy": (None, [ctypes.c_void_p]),
    "pic_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pic_params), ctypes.c_uint64]),
    "pic_deposit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "poisson_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                     ctypes.c_int]),
    "poisson_solve_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                        ctypes.c_int, ctypes.POINTER(pic_solve_opts),
                                        ctypes.POINTER(pic_solve_info)]),
    "pic_gather_push": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    "pic_sync_velocity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    "pic_field_energy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "pic_get_particles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]),
    "pic_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int]),
    "pic_set_particles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "pic_num_particles": (ctypes.c_int64, [ctypes.c_void_p]),
    "pic_apply_laplacian": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pic_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pic_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "pic_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pic_profile_stats), ctypes.c_int]),
    "pic_cnn_set_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pic_cnn_get_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pic_cnn_get_grads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pic_cnn_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pic_cnn_set_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "pic_mg_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "pic_fft_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pic_ssor_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pic_pif_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]),
    "pic_pif_push": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]),
    "pic_gather_push_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    "pic_sync_velocity_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    "pic_field_energy_E": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "pic_cnn_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_int]),
    "pic_cnn_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "pic_cnn_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "pic_cnn_make_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_double]),
    "pic_cnn_loss": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "pic_cnn_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pic_train_opts), ctypes.POINTER(pic_train_info)]),
    "pic_cnn_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "pic_cnn_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "pic_cnn_set_train_precision": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "pic_cnn_conv_raw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_int]),
    "pic_field_energy_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                                ctypes.c_void_p]),
}


def lib():
    """The loaded libpic.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2605_05469_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def strerror(code):
    try:
        return lib().pic_strerror(code).decode()
    except ImportError:
        return f"error {code}"


def _check(code, what):
    if code != PIC_OK:
        raise PicError(code, what)
    return code


def _dptr(t, dtype_name, numel, what):
    """Device pointer of a contiguous CUDA tensor of the given dtype and size."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what}: expected a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}" or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{what}: expected a contiguous {dtype_name} tensor with {numel} elements, "
                         f"got {t.dtype} {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ------------------------------------------------------------ C-named calls
def pic_create(stream=None):
    h = ctypes.c_void_p()
    _check(lib().pic_create(ctypes.byref(h), _stream_ptr(stream)), "pic_create")
    return h


def pic_destroy(h):
    lib().pic_destroy(h)


def pic_init(h, N, ppc, seed, alpha=0.05, k=0.5, vth=1.0, init_mode=0):
    p = pic_params(N, ppc, alpha, k, vth, init_mode)
    _check(lib().pic_init(h, ctypes.byref(p), ctypes.c_uint64(seed)), "pic_init")


def pic_deposit(h, rho, n):
    _check(lib().pic_deposit(h, _dptr(rho, "float64", n, "rho")), "pic_deposit")


def poisson_solve(h, rho, phi, tol, maxit, n):
    return lib().poisson_solve(h, _dptr(rho, "float64", n, "rho"), _dptr(phi, "float64", n, "phi"), tol, maxit)


def poisson_solve_ex(h, rho, phi, tol, maxit, n, precision=PREC_FP64, precond=PC_JACOBI, reliable_delta=0.0,
                     check_every=0, refine_max=0):
    o = pic_solve_opts(precision, precond, reliable_delta, check_every, refine_max)
    info = pic_solve_info()
    code = lib().poisson_solve_ex(h, _dptr(rho, "float64", n, "rho"), _dptr(phi, "float64", n, "phi"), tol, maxit,
                                  ctypes.byref(o), ctypes.byref(info))
    return code, info.as_dict()


def pic_gather_push(h, phi, dt, n):
    _check(lib().pic_gather_push(h, _dptr(phi, "float64", n, "phi"), dt), "pic_gather_push")


def pic_sync_velocity(h, phi, dt, n):
    _check(lib().pic_sync_velocity(h, _dptr(phi, "float64", n, "phi"), dt), "pic_sync_velocity")


def pic_field_energy(h, phi, n):
    out = (ctypes.c_double * 3)()
    _check(lib().pic_field_energy(h, _dptr(phi, "float64", n, "phi"), out), "pic_field_energy")
    return np.array(list(out))


def pic_get_particles(h, np_):
    out = np.empty(6 * np_, dtype=np.float64)
    half = ctypes.c_int()
    _check(lib().pic_get_particles(h, out.ctypes.data_as(ctypes.c_void_p), 0, ctypes.byref(half)),
           "pic_get_particles")
    return out.reshape(6, np_), bool(half.value)


def pic_apply_laplacian(h, x, y, n):
    _check(lib().pic_apply_laplacian(h, _dptr(x, "float64", n, "x"), _dptr(y, "float64", n, "y")),
           "pic_apply_laplacian")


def pic_profile_enable(h, on=True):
    _check(lib().pic_profile_enable(h, 1 if on else 0), "pic_profile_enable")


def pic_profile_read(h, reset=True):
    st = pic_profile_stats()
    _check(lib().pic_profile_read(h, ctypes.byref(st), 1 if reset else 0), "pic_profile_read")
    return st.as_dict()


def pic_field_energy_noalloc(phi, N, k, out_w, stream=None):
    """Field energy into the device tensor out_w (3 float64) without any
    allocation inside the library (see include/pic.h); returns the status code."""
    return lib().pic_field_energy_noalloc(_dptr(phi, "float64", N ** 3, "phi"), N, k,
                                          _dptr(out_w, "float64", 3, "out_w"), _stream_ptr(stream))


# ------------------------------------------------------------ convenience
class Context:
    """One PIC problem on the current CUDA device (owns particles and workspace)."""

    def __init__(self, stream=None):
        self.h = pic_create(stream)
        self.N = 0
        self.n = 0

    def init(self, N, ppc, seed, alpha=0.05, k=0.5, vth=1.0, init_mode=0):
        pic_init(self.h, N, ppc, seed, alpha, k, vth, init_mode)
        self.N, self.n = N, N ** 3
        self.L = 2.0 * np.pi / k
        self.h_grid = self.L / N
        return self

    @property
    def num_particles(self):
        return int(lib().pic_num_particles(self.h))

    def deposit(self, rho):
        pic_deposit(self.h, rho, self.n)

    def solve(self, rho, phi, tol=1e-10, maxit=5000, precision=PREC_FP64, precond=PC_JACOBI, reliable_delta=0.0,
              check_every=0, raise_on_error=True, refine_max=0):
        code, info = poisson_solve_ex(self.h, rho, phi, tol, maxit, self.n, precision, precond, reliable_delta,
                                      check_every, refine_max)
        info["code"] = code
        if raise_on_error and code not in (PIC_OK,):
            raise PicError(code, "poisson_solve_ex")
        return info

    def gather_push(self, phi, dt):
        pic_gather_push(self.h, phi, dt, self.n)

    def sync_velocity(self, phi, dt):
        pic_sync_velocity(self.h, phi, dt, self.n)

    def field_energy(self, phi):
        return pic_field_energy(self.h, phi, self.n)

    def pif_field(self, E, tol=1e-12):
        """The particle-in-Fourier field at the particles, E [3 Np] in the original order."""
        _check(lib().pic_pif_field(self.h, tol, _dptr(E, "float64", 3 * self.num_particles, "E")), "pic_pif_field")

    def pif_push(self, dt, tol=1e-12):
        _check(lib().pic_pif_push(self.h, tol, dt), "pic_pif_push")

    def ssor_apply(self, r, z):
        """z = M r of the red-black SSOR preconditioner (FP32, scaled units)."""
        _check(lib().pic_ssor_apply(self.h, _dptr(r, "float32", self.n, "r"), _dptr(z, "float32", self.n, "z")),
               "pic_ssor_apply")

    def fft_solve(self, rho, phi, E=None):
        """FFT pseudo-spectral solve: phi (and E [3 N^3] if given) from rho."""
        _check(lib().pic_fft_solve(self.h, _dptr(rho, "float64", self.n, "rho"), _dptr(phi, "float64", self.n, "phi"),
                                   None if E is None else _dptr(E, "float64", 3 * self.n, "E")), "pic_fft_solve")

    def gather_push_field(self, E, dt):
        _check(lib().pic_gather_push_field(self.h, _dptr(E, "float64", 3 * self.n, "E"), dt), "pic_gather_push_field")

    def sync_velocity_field(self, E, dt):
        _check(lib().pic_sync_velocity_field(self.h, _dptr(E, "float64", 3 * self.n, "E"), dt),
               "pic_sync_velocity_field")

    def field_energy_E(self, E):
        out = (ctypes.c_double * 3)()
        _check(lib().pic_field_energy_E(self.h, _dptr(E, "float64", 3 * self.n, "E"), out), "pic_field_energy_E")
        return np.array(list(out))

    def particles(self):
        return pic_get_particles(self.h, self.num_particles)

    def particles_into(self, out):
        """The particles into a device FP64 tensor of 6 Np (x, y, z, vx, vy, vz
        blocks, original order); returns whether velocities lag by dt/2."""
        half = ctypes.c_int()
        _check(lib().pic_get_particles(self.h, _dptr(out, "float64", 6 * self.num_particles, "out"), 1,
                                       ctypes.byref(half)), "pic_get_particles")
        return bool(half.value)

    def selftest_bounded_wait(self, budget_ns, producer):
        """Status code of the bounded-wait self-test (PIC_OK or PIC_ETIMEOUT)."""
        return lib().pic_selftest_bounded_wait(self.h, int(budget_ns), 1 if producer else 0)

    def particles_to_host(self, out):
        """The particles into a host FP64 tensor of 6 Np (pinned or pageable; x,
        y, z, vx, vy, vz blocks, original order); returns whether velocities lag
        by dt/2."""
        import torch
        if not isinstance(out, torch.Tensor) or out.is_cuda or out.dtype != torch.float64 or \
                not out.is_contiguous() or out.numel() != 6 * self.num_particles:
            raise ValueError("out: expected a contiguous host float64 tensor of 6 Np elements")
        half = ctypes.c_int()
        _check(lib().pic_get_particles(self.h, ctypes.c_void_p(out.data_ptr()), 0, ctypes.byref(half)),
               "pic_get_particles")
        return bool(half.value)

    def set_particles(self, state, half_step):
        """Replace the particle state by a FP64 tensor of 6 Np (x, y, z, vx, vy,
        vz blocks), on the device or on the host; `half_step`: velocities lag
        the positions by dt/2."""
        import torch
        if isinstance(state, np.ndarray):
            state = torch.from_numpy(np.ascontiguousarray(state, dtype=np.float64).reshape(-1))
        if not isinstance(state, torch.Tensor) or state.dtype != torch.float64 or not state.is_contiguous() or \
                state.numel() != 6 * self.num_particles:
            raise ValueError("state: expected a contiguous float64 tensor of 6 Np elements")
        _check(lib().pic_set_particles(self.h, ctypes.c_void_p(state.data_ptr()), 1 if state.is_cuda else 0,
                                       1 if half_step else 0), "pic_set_particles")

    def apply_laplacian(self, x, y):
        pic_apply_laplacian(self.h, x, y, self.n)

    def residual(self, rho, phi, r):
        _check(lib().pic_residual(self.h, _dptr(rho, "float64", self.n, "rho"), _dptr(phi, "float64", self.n, "phi"),
                                  _dptr(r, "float64", self.n, "r")), "pic_residual")

    # ---- learned preconditioner
    def cnn_set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32).reshape(-1)
        if w.size != CNN_WEIGHTS:
            raise ValueError(f"expected {CNN_WEIGHTS} weights, got {w.size}")
        _check(lib().pic_cnn_set_weights(self.h, w.ctypes.data_as(ctypes.c_void_p)), "pic_cnn_set_weights")

    def cnn_get_weights(self):
        w = np.empty(CNN_WEIGHTS, dtype=np.float32)
        _check(lib().pic_cnn_get_weights(self.h, w.ctypes.data_as(ctypes.c_void_p)), "pic_cnn_get_weights")
        return w

    def cnn_get_grads(self):
        g = np.empty(CNN_WEIGHTS, dtype=np.float32)
        _check(lib().pic_cnn_get_grads(self.h, g.ctypes.data_as(ctypes.c_void_p)), "pic_cnn_get_grads")
        return g

    def mg_apply(self, r, z, learned=False):
        _check(lib().pic_mg_apply(self.h, _dptr(r, "float32", self.n, "r"), _dptr(z, "float32", self.n, "z"),
                                  1 if learned else 0), "pic_mg_apply")

    def cnn_set_apply(self, mode):
        _check(lib().pic_cnn_set_apply(self.h, int(mode)), "pic_cnn_set_apply")
        return self

    def cnn_apply(self, r, z):
        _check(lib().pic_cnn_apply(self.h, _dptr(r, "float32", self.n, "r"), _dptr(z, "float32", self.n, "z")),
               "pic_cnn_apply")

    def cnn_train(self, target=TRAIN_PRECONDITIONER, grid=64, sets=4, steps=600, batch=8, crop=32, lr=2e-3,
                  seed=11, validate_every=100, val_grid=128, val_seed=21, resume=False, restarts=1,
                  raise_on_error=True):
        """pic_cnn_train: trains the network in the library and keeps the
        result in this context; returns the training info (and its code)."""
        o = pic_train_opts(int(target), grid, sets, steps, batch, crop, lr, seed, validate_every, val_grid, val_seed,
                           1 if resume else 0, restarts)
        info = pic_train_info()
        code = lib().pic_cnn_train(self.h, ctypes.byref(o), ctypes.byref(info))
        if raise_on_error:
            _check(code, "pic_cnn_train")
        d = info.as_dict()
        d["code"] = code
        return d

    def cnn_save(self, path):
        _check(lib().pic_cnn_save(self.h, os.fsencode(path)), "pic_cnn_save")

    def cnn_load(self, path):
        _check(lib().pic_cnn_load(self.h, os.fsencode(path)), "pic_cnn_load")

    def cnn_set_train_precision(self, mode):
        _check(lib().pic_cnn_set_train_precision(self.h, int(mode)), "pic_cnn_set_train_precision")
        return self

    def cnn_forward(self, x, y, B, D):
        n = B * D ** 3
        _check(lib().pic_cnn_forward(self.h, _dptr(x, "float32", n, "x"), _dptr(y, "float32", n, "y"), B, D),
               "pic_cnn_forward")

    def cnn_backward(self, gy, B, D):
        _check(lib().pic_cnn_backward(self.h, _dptr(gy, "float32", B * D ** 3, "gy"), B, D), "pic_cnn_backward")

    def cnn_adam(self, lr):
        _check(lib().pic_cnn_adam(self.h, lr), "pic_cnn_adam")

    def cnn_make_batch(self, r, a, b, origins, D, x, t, h2):
        o = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1)
        B = o.size // 3
        n, m = self.n, B * D ** 3
        _check(lib().pic_cnn_make_batch(self.h, _dptr(r, "float64", n, "r"), _dptr(a, "float64", n, "a"),
                                        _dptr(b, "float64", n, "b"), o.ctypes.data_as(ctypes.c_void_p), B, D,
                                        _dptr(x, "float32", m, "x"), _dptr(t, "float32", m, "t"), h2),
               "pic_cnn_make_batch")

    def cnn_loss(self, y, t, B, D, gy):
        m = B * D ** 3
        loss = ctypes.c_double()
        _check(lib().pic_cnn_loss(self.h, _dptr(y, "float32", m, "y"), _dptr(t, "float32", m, "t"), B, D,
                                  _dptr(gy, "float32", m, "gy"), ctypes.byref(loss)), "pic_cnn_loss")
        return loss.value

    def cnn_conv_raw(self, which, x, out, B, D):
        import torch
        m = B * D ** 3
        if which in (0, 4):
            px = _dptr(x, "float32", m, "x")
        else:
            px = _dptr(x, "bfloat16", 16 * m, "x")
        _check(lib().pic_cnn_conv_raw(self.h, which, px, _dptr(out, "float32", 16 * m, "out"), B, D),
               "pic_cnn_conv_raw")

    def profile(self, on=True):
        pic_profile_enable(self.h, on)

    def profile_read(self, reset=True):
        return pic_profile_read(self.h, reset)

    def close(self):
        if self.h is not None:
            pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
