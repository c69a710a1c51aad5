"""ctypes wrapper of the CPU oracle (oracle/liboracle.so).

TEST INFRASTRUCTURE ONLY: the plain CPU reference for the particle-learning
cycle of arXiv 1212.1639.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import this module.  It never imports the
product package and the product package never imports it.
"""
import ctypes as C
import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


class OrConfig(C.Structure):
    _fields_ = [("n", C.c_uint64), ("seed", C.c_uint64), ("filter_id", C.c_uint32),
                ("scheme", C.c_int32), ("precision", C.c_int32),
                ("known_variances", C.c_int32),
                ("x0_mean", C.c_double), ("x0_var", C.c_double),
                ("a_sigma", C.c_double), ("b_sigma", C.c_double),
                ("a_tau", C.c_double), ("b_tau", C.c_double),
                ("sigma2", C.c_double), ("tau2", C.c_double), ("algorithm", C.c_int32),
                ("ess_frac", C.c_double)]


PARTICLE_LEARNING, BOOTSTRAP = 0, 1


def _declare(L):
    V, I, U32, U64, D = None, C.c_int, C.c_uint32, C.c_uint64, C.c_double
    sig = {
        "or_philox4x32": (V, [u32p, u32p, u32p, U64]),
        "or_philox4x64": (V, [u64p, u64p, u64p, U64]),
        "or_draw": (V, [U64, U32, U32, U32, U32, U32, U32, u32p]),
        "or_unif_f32": (V, [u32p, U64, f32p]),
        "or_det_log_f32": (V, [f32p, f32p, U64]),
        "or_det_log_f64": (V, [f64p, f64p, U64]),
        "or_det_exp_core_f32": (V, [f32p, f32p, U64]),
        "or_det_exp_core_f64": (V, [f64p, f64p, U64]),
        "or_det_cos2pi_f32": (V, [f32p, f32p, U64]),
        "or_det_cos2pi_f64": (V, [f64p, f64p, U64]),
        "or_det_sincos2pi_f32": (V, [f32p, f32p, f32p, U64]),
        "or_det_sincos2pi_f64": (V, [f64p, f64p, f64p, U64]),
        "or_quant_exp_f32": (V, [f32p, U64, I, u64p, f32p]),
        "or_quant_exp_f64": (V, [f64p, U64, I, u64p, f64p]),
        "or_normals_f32": (V, [U64, U32, U32, U32, U64, f32p]),
        "or_normals_f64": (V, [U64, U32, U32, U32, U64, f64p]),
        "or_theta_draws_f32": (V, [U64, U32, U32, U64, f32p]),
        "or_theta_draws_f64": (V, [U64, U32, U32, U64, f64p]),
        "or_gamma_f32": (I, [D, U64, U32, U32, U32, U64, f32p]),
        "or_gamma_f64": (I, [D, U64, U32, U32, U32, U64, f64p]),
        "or_mt_constants": (V, [D, f64p]),
        "or_cdf_shift": (I, [U64]),
        "or_cdf_scan": (V, [u64p, U64, u64p]),
        "or_quantize_weights_f32": (I, [f32p, U64, u64p]),
        "or_systematic_offset": (U64, [U64, U64, U32, U32]),
        "or_stratified_offset": (U64, [U64, U64, U32, U32, U64]),
        "or_spacing_prefix": (V, [U64, U64, U32, U32, u64p]),
        "or_resample_method": (V, [u64p, U64, I, I, U64, U32, U32, u32p]),
        "or_systematic_with_offset": (V, [u64p, U64, U64, u32p]),
        "or_cutpoint_search": (V, [u64p, U64, u64p, u32p]),
        "or_cutpoint_method_int": (V, [u64p, U64, u32p, u64p, U64, u32p, u64p]),
        "or_resample_cdf": (V, [u64p, U64, I, U64, U32, U32, u32p]),
        "or_resample_weights": (I, [f32p, U64, I, U64, U32, U32, u32p]),
        "or_pl_create": (C.c_void_p, [C.POINTER(OrConfig)]),
        "or_pl_resampled": (I, [C.c_void_p]),
        "or_ess_resample": (I, [u64p, U64, D]),
        "or_pl_step": (I, [C.c_void_p, D]),
        "or_pl_estimate": (V, [C.c_void_p, f64p]),
        "or_pl_state": (V, [C.c_void_p, f64p, f64p, f64p, f64p, f64p]),
        "or_pl_state_raw": (V, [C.c_void_p] + [C.c_void_p] * 5),
        "or_pl_ancestors": (V, [C.c_void_p, u32p]),
        "or_pl_cdf": (V, [C.c_void_p, u64p]),
        "or_pl_destroy": (V, [C.c_void_p]),
        "or_suffstat_known_states": (I, [C.POINTER(OrConfig), f64p, f64p, U32,
                                         f64p, f64p, f64p, f64p]),
        "or_kalman": (V, [f64p, U32, D, D, D, D, f64p, f64p, f64p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


# Purposes of the counter-based draws (fourth counter word, low byte).
P_INIT_X, P_INIT_SIGMA, P_INIT_TAU = 1, 2, 3
P_STATE, P_GAMMA_SIGMA, P_GAMMA_TAU = 4, 5, 6
P_SYS_OFFSET, P_SPACING = 7, 8

MULTINOMIAL, SYSTEMATIC, MULTINOMIAL_CUTPOINT, SYSTEMATIC_CUTPOINT, STRATIFIED = 0, 1, 2, 3, 4
FP32, FP64 = 0, 1


def philox4x32(ctr, key):
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    lib().or_philox4x32(ctr, key, out, ctr.shape[0])
    return out


def philox4x64(ctr, key):
    ctr = np.ascontiguousarray(ctr, np.uint64).reshape(-1, 4)
    key = np.ascontiguousarray(key, np.uint64).reshape(-1, 2)
    out = np.zeros_like(ctr)
    lib().or_philox4x64(ctr, key, out, ctr.shape[0])
    return out


def draws(seed, filt, t, j0, count, purpose, attempt=0):
    out = np.zeros((count, 4), np.uint32)
    lib().or_draw(seed, filt, t, j0, count, purpose, attempt, out)
    return out


def unif_f32(w):
    w = np.ascontiguousarray(w, np.uint32)
    out = np.zeros(w.shape, np.float32)
    lib().or_unif_f32(w, w.size, out)
    return out


def _vec(name, x, dtype):
    x = np.ascontiguousarray(x, dtype)
    out = np.zeros_like(x)
    getattr(lib(), name)(x, out, x.size)
    return out


def det_log(x, dtype=np.float32):
    return _vec("or_det_log_f32" if dtype == np.float32 else "or_det_log_f64", x, dtype)


def det_exp_core(x, dtype=np.float32):
    return _vec("or_det_exp_core_f32" if dtype == np.float32 else "or_det_exp_core_f64", x, dtype)


def det_cos2pi(x, dtype=np.float32):
    return _vec("or_det_cos2pi_f32" if dtype == np.float32 else "or_det_cos2pi_f64", x, dtype)


def det_sincos2pi(x, dtype=np.float32):
    x = np.ascontiguousarray(x, dtype)
    s = np.zeros_like(x)
    c = np.zeros_like(x)
    f = lib().or_det_sincos2pi_f32 if dtype == np.float32 else lib().or_det_sincos2pi_f64
    f(x, s, c, x.size)
    return s, c


def quant_exp(dl, k, dtype=np.float32):
    dl = np.ascontiguousarray(dl, dtype)
    W = np.zeros(dl.size, np.uint64)
    e = np.zeros(dl.size, dtype)
    f = lib().or_quant_exp_f32 if dtype == np.float32 else lib().or_quant_exp_f64
    f(dl, dl.size, k, W, e)
    return W, e


def normals(seed, filt, t, purpose, n, dtype=np.float32):
    out = np.zeros(n, dtype)
    f = lib().or_normals_f32 if dtype == np.float32 else lib().or_normals_f64
    f(seed, filt, t, purpose, n, out)
    return out


def theta_draws(seed, filt, t, n, dtype=np.float32):
    """The propagation draws of slots 0..n-1 at cycle t: columns Zx, Zs, Us, Zt, Ut."""
    out = np.zeros((n, 5), dtype)
    f = lib().or_theta_draws_f32 if dtype == np.float32 else lib().or_theta_draws_f64
    f(seed, filt, t, n, out)
    return out


def mt_constants(a):
    """(d, c, K) of the Marsaglia-Tsang sampler for shape a, in binary64."""
    out = np.zeros(3, np.float64)
    lib().or_mt_constants(float(a), out)
    return float(out[0]), float(out[1]), float(out[2])


def gammas(a, seed, filt, t, purpose, n, dtype=np.float32):
    out = np.zeros(n, dtype)
    f = lib().or_gamma_f32 if dtype == np.float32 else lib().or_gamma_f64
    fail = f(a, seed, filt, t, purpose, n, out)
    return out, fail


def cdf_shift(n):
    return lib().or_cdf_shift(n)


def cdf_scan(W):
    W = np.ascontiguousarray(W, np.uint64)
    Q = np.zeros_like(W)
    lib().or_cdf_scan(W, W.size, Q)
    return Q


def quantize_weights(w):
    w = np.ascontiguousarray(w, np.float32)
    W = np.zeros(w.size, np.uint64)
    rc = lib().or_quantize_weights_f32(w, w.size, W)
    if rc != 0:
        raise ValueError("invalid weights")
    return W


def systematic_offset(T, seed, filt, t):
    return lib().or_systematic_offset(T, seed, filt, t)


def stratified_offset(T, seed, filt, t, j):
    return lib().or_stratified_offset(T, seed, filt, t, j)


def spacing_prefix(n, seed, filt, t):
    S = np.zeros(n + 1, np.uint64)
    lib().or_spacing_prefix(n, seed, filt, t, S)
    return S


def resample_method(Q, positions, method, seed, filt, t):
    """positions: 'multinomial' | 'systematic' | 'stratified'; method: 'walk' | 'naive' |
    'cutpoint'."""
    Q = np.ascontiguousarray(Q, np.uint64)
    anc = np.zeros(Q.size, np.uint32)
    lib().or_resample_method(Q, Q.size, {"multinomial": 0, "systematic": 1, "stratified": 2}[positions],
                             {"walk": 0, "naive": 1, "cutpoint": 2}[method],
                             seed, filt, t, anc)
    return anc


def systematic_with_offset(Q, r):
    Q = np.ascontiguousarray(Q, np.uint64)
    anc = np.zeros(Q.size, np.uint32)
    lib().or_systematic_with_offset(Q, Q.size, r, anc)
    return anc


def cutpoint_search(Q):
    Q = np.ascontiguousarray(Q, np.uint64)
    L = np.zeros(Q.size, np.uint64)
    I = np.zeros(Q.size, np.uint32)
    lib().or_cutpoint_search(Q, Q.size, L, I)
    return L, I


def cutpoint_method_int(Q, I, U):
    Q = np.ascontiguousarray(Q, np.uint64)
    I = np.ascontiguousarray(I, np.uint32)
    U = np.ascontiguousarray(U, np.uint64)
    anc = np.zeros(U.size, np.uint32)
    bucket = np.zeros(U.size, np.uint64)
    lib().or_cutpoint_method_int(Q, Q.size, I, U, U.size, anc, bucket)
    return anc, bucket


def resample_cdf(Q, scheme, seed, filt, t):
    Q = np.ascontiguousarray(Q, np.uint64)
    anc = np.zeros(Q.size, np.uint32)
    lib().or_resample_cdf(Q, Q.size, scheme, seed, filt, t, anc)
    return anc


def resample_weights(w, scheme, seed, filt, t):
    """Ancestors for FP32 weights w (the semantics of pf_resample)."""
    w = np.ascontiguousarray(w, np.float32)
    anc = np.zeros(w.size, np.uint32)
    rc = lib().or_resample_weights(w, w.size, scheme, seed, filt, t, anc)
    if rc != 0:
        raise ValueError("invalid weights")
    return anc


def make_config(n, seed=1212, filter_id=0, scheme=MULTINOMIAL, precision=FP64,
                x0_mean=0.0, x0_var=10.0, a_sigma=3.0, b_sigma=2.0, a_tau=3.0, b_tau=2.0,
                known_variances=False, sigma2=1.0, tau2=0.1, algorithm=PARTICLE_LEARNING,
                ess_frac=0.0):
    """algorithm: PARTICLE_LEARNING or BOOTSTRAP (Algorithm "Particle Filtering",
    which takes the variances as known).  ess_frac > 0: adaptive resampling
    (particle learning only), see oracle.h."""
    if algorithm == BOOTSTRAP and not known_variances:
        raise ValueError("the bootstrap filter takes known variances")
    return OrConfig(n=n, seed=seed, filter_id=filter_id, scheme=scheme, precision=precision,
                    known_variances=int(known_variances), x0_mean=x0_mean, x0_var=x0_var,
                    a_sigma=a_sigma, b_sigma=b_sigma, a_tau=a_tau, b_tau=b_tau,
                    sigma2=sigma2, tau2=tau2, algorithm=int(algorithm), ess_frac=float(ess_frac))


ESTIMATE_FIELDS = ("t", "x_mean", "x_var", "sigma2_mean", "sigma2_var",
                   "tau2_mean", "tau2_var", "log_marglik")


class Filter:
    """One particle-learning filter on the CPU (FP32 or FP64 state)."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.n = cfg.n
        self.h = lib().or_pl_create(C.byref(cfg))

    def step(self, y):
        rc = lib().or_pl_step(self.h, float(y))
        if rc != 0:
            raise RuntimeError("oracle step failed with status %d" % rc)

    def run(self, ys):
        for y in ys:
            self.step(y)

    def estimate(self):
        out = np.zeros(8, np.float64)
        lib().or_pl_estimate(self.h, out)
        return dict(zip(ESTIMATE_FIELDS, out.tolist()))

    def state(self):
        arrs = [np.zeros(self.n, np.float64) for _ in range(5)]
        lib().or_pl_state(self.h, *arrs)
        return dict(zip(("x", "sigma2", "tau2", "b_sigma", "b_tau"), arrs))

    def state_raw(self):
        rt = np.float32 if self.cfg.precision == FP32 else np.float64
        bt = np.uint64 if self.cfg.precision == FP32 else np.float64
        arrs = [np.zeros(self.n, rt) for _ in range(3)] + [np.zeros(self.n, bt) for _ in range(2)]
        lib().or_pl_state_raw(self.h, *[a.ctypes.data for a in arrs])
        return dict(zip(("x", "sigma2", "tau2", "b_sigma", "b_tau"), arrs))

    def ancestors(self):
        a = np.zeros(self.n, np.uint32)
        lib().or_pl_ancestors(self.h, a)
        return a

    def resampled(self):
        """Whether the last cycle resampled (always, unless adaptive)."""
        return bool(lib().or_pl_resampled(self.h))

    def cdf(self):
        q = np.zeros(self.n, np.uint64)
        lib().or_pl_cdf(self.h, q)
        return q

    def close(self):
        if self.h:
            lib().or_pl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def suffstat_known_states(cfg, xpath, y):
    xpath = np.ascontiguousarray(xpath, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    T = y.size
    assert xpath.size == T + 1
    outs = [np.zeros(cfg.n, np.float64) for _ in range(4)]
    rc = lib().or_suffstat_known_states(C.byref(cfg), xpath, y, T, *outs)
    return dict(zip(("b_sigma", "b_tau", "sigma2", "tau2"), outs)), rc


def ess_resample(W, ess_frac):
    """The adaptive resampling decision for quantised weights W (uint64)."""
    W = np.ascontiguousarray(W, np.uint64)
    return bool(lib().or_ess_resample(W, W.size, float(ess_frac)))


def kalman(y, m0, P0, sigma2, tau2):
    y = np.ascontiguousarray(y, np.float64)
    mean = np.zeros(y.size)
    var = np.zeros(y.size)
    ll = np.zeros(1)
    lib().or_kalman(y, y.size, m0, P0, sigma2, tau2, mean, var, ll)
    return mean, var, float(ll[0])
