"""Python binding of the l1ls C ABI (``include/l1ls.h``): argument marshalling only.

Every step of generation, products and solves runs in the CUDA library ``libl1ls.so``;
this module only converts arguments.  Importing it loads the library and raises if it is
missing -- there is no fallback path.  Vectors may be CUDA ``torch`` tensors (used in
place, work enqueued on the given stream) or numpy arrays / CPU tensors (staged by the
library, the call returns when the result is on the host).
"""

import ctypes
import math
import os

import numpy as np

__all__ = ["Context", "Instance", "L1LSError", "lib", "library_path", "F64", "F32", "BF16"]

F64, F32, BF16 = 0, 1, 2
_DTYPES = {"f64": F64, "f32": F32, "bf16": BF16, F64: F64, F32: F32, BF16: BF16}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOCONV", 6: "ENUMERIC",
          7: "EBUSY", 8: "ENOTFOUND", 9: "ECANCELLED"}


class GenParams(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64), ("n", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("kappa", ctypes.c_double), ("tau", ctypes.c_double), ("xstar_frac", ctypes.c_double),
                ("xstar_lo", ctypes.c_double), ("xstar_hi", ctypes.c_double), ("theta", ctypes.c_double),
                ("vartheta", ctypes.c_double), ("right_stages", ctypes.c_int32), ("left_stages", ctypes.c_int32),
                ("value_dtype", ctypes.c_int32), ("g_offsupport", ctypes.c_int32),
                ("n_nnz_per_col", ctypes.c_int32), ("matrix_free", ctypes.c_int32),
                ("sigma_mode", ctypes.c_int32), ("xstar_mode", ctypes.c_int32), ("sigma_odd", ctypes.c_double),
                ("sigma_even", ctypes.c_double), ("gamma", ctypes.c_double)]


class InstInfo(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64), ("n", ctypes.c_uint64), ("nnz", ctypes.c_uint64), ("s", ctypes.c_uint64),
                ("f_star", ctypes.c_double), ("lipschitz", ctypes.c_double), ("lam_max", ctypes.c_double),
                ("tau_gen", ctypes.c_double), ("value_dtype", ctypes.c_int32), ("right_stages", ctypes.c_int32),
                ("left_stages", ctypes.c_int32), ("igen2", ctypes.c_int32), ("matrix_free", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("device_bytes", ctypes.c_uint64)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("rel_gap_tol", ctypes.c_double), ("max_iter", ctypes.c_int64),
                ("time_limit_s", ctypes.c_double), ("mu", ctypes.c_double), ("mu_min", ctypes.c_double),
                ("mu_start", ctypes.c_double), ("pcg_rtol", ctypes.c_double), ("armijo", ctypes.c_double), ("ls_max", ctypes.c_int32),
                ("pcg_max", ctypes.c_int32), ("check_every", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("accum", ctypes.c_int32), ("f_target", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("products", ctypes.c_int64), ("cg_iters", ctypes.c_int64),
                ("ls_trials", ctypes.c_int64), ("f", ctypes.c_double), ("dual", ctypes.c_double),
                ("gap", ctypes.c_double), ("rel_gap", ctypes.c_double), ("seconds", ctypes.c_double),
                ("mu", ctypes.c_double), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("queue_s", ctypes.c_double), ("latency_s", ctypes.c_double), ("L", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}
        d["status_name"] = STATUS.get(self.status, str(self.status))
        return d


class ServeInfo(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("running", ctypes.c_int32), ("peak_running", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("completed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("capacity_bytes", ctypes.c_uint64), ("reserved_bytes", ctypes.c_uint64),
                ("peak_reserved_bytes", ctypes.c_uint64)]


FISTA, PDNCG = 0, 1
METHODS = {"fista": FISTA, "pdncg": PDNCG}


class L1LSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


library_path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libl1ls.so")

if not os.path.exists(library_path):
    raise ImportError("libl1ls.so is not built (%s); run __graft_entry__.build() or "
                      "python paper_1503_03520_gb300/_build.py" % library_path)

lib = ctypes.CDLL(library_path)

_P = ctypes.c_void_p
_sig = {
    "l1ls_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "l1ls_destroy": (ctypes.c_int, [_P]),
    "l1ls_generate": (ctypes.c_int, [_P, ctypes.POINTER(GenParams), _P, ctypes.POINTER(_P)]),
    "l1ls_inst_free": (ctypes.c_int, [_P]),
    "l1ls_inst_get_info": (ctypes.c_int, [_P, ctypes.POINTER(InstInfo)]),
    "l1ls_inst_kappa_rho": (ctypes.c_int, [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "l1ls_inst_export": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "l1ls_inst_export_t": (ctypes.c_int, [_P, _P, _P, _P]),
    "l1ls_matvec": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    "l1ls_rmatvec": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    "l1ls_rmatvec_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    "l1ls_solve_fista": (ctypes.c_int, [_P, ctypes.POINTER(SolveOpts), _P, _P, ctypes.POINTER(Result), _P]),
    "l1ls_solve_fista_bt": (ctypes.c_int, [_P, ctypes.POINTER(SolveOpts), ctypes.c_double, ctypes.c_double, _P, _P,
                                           ctypes.POINTER(Result), _P]),
    "l1ls_solve_pdncg": (ctypes.c_int, [_P, ctypes.POINTER(SolveOpts), _P, _P, ctypes.POINTER(Result), _P]),
    "l1ls_fista_begin": (ctypes.c_int, [_P, ctypes.POINTER(SolveOpts), _P, _P]),
    "l1ls_fista_step": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P]),
    "l1ls_fista_end": (ctypes.c_int, [_P, _P, ctypes.POINTER(Result), _P]),
    "l1ls_batch_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "l1ls_batch_solve_path": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                             ctypes.POINTER(SolveOpts), _P, _P, _P]),
    "l1ls_batch_get_schedule": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_double)]),
    "l1ls_batch_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
    "l1ls_batch_free": (ctypes.c_int, [_P]),
    "l1ls_batch_barrier_selftest": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)]),
    "l1ls_footprint": (ctypes.c_size_t, [ctypes.POINTER(GenParams), ctypes.c_int]),
    "l1ls_serve_config": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_size_t]),
    "l1ls_submit": (ctypes.c_int, [_P, ctypes.POINTER(GenParams), ctypes.POINTER(SolveOpts), ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_uint64)]),
    "l1ls_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(Result), _P]),
    "l1ls_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "l1ls_serve_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServeInfo)]),
    "l1ls_gen_params_default": (None, [ctypes.POINTER(GenParams)]),
    "l1ls_solve_opts_default": (None, [ctypes.POINTER(SolveOpts)]),
    "l1ls_last_error": (ctypes.c_char_p, []),
    "l1ls_version": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _check(status, allow=()):
    if status != 0 and status not in allow:
        raise L1LSError(status, lib.l1ls_last_error().decode())
    return status


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _vec_ptr(v):
    """(pointer, dtype code, keepalive) for a torch tensor or numpy array."""
    try:
        import torch
        if isinstance(v, torch.Tensor):
            if not v.is_contiguous():
                raise ValueError("vector must be contiguous")
            code = {torch.float64: F64, torch.float32: F32}.get(v.dtype)
            if code is None:
                raise ValueError("vector dtype must be float64 or float32")
            return ctypes.c_void_p(v.data_ptr()), code, v
    except ImportError:
        pass
    a = np.ascontiguousarray(v)
    code = {np.dtype(np.float64): F64, np.dtype(np.float32): F32}.get(a.dtype)
    if code is None:
        raise ValueError("vector dtype must be float64 or float32")
    return ctypes.c_void_p(a.ctypes.data), code, a


def _numel(v):
    n = getattr(v, "numel", None)
    if callable(n):
        return int(n())
    return int(np.asarray(v).size)


def gen_params(d):
    """GenParams from a parameter dict (keys of ``l1ls_gen_params``; value_dtype may be a name)."""
    p = GenParams()
    lib.l1ls_gen_params_default(ctypes.byref(p))
    for k, v in d.items():
        if k == "value_dtype":
            v = _DTYPES[v]
        if hasattr(p, k):
            setattr(p, k, v)
    return p


def solve_opts(**kw):
    o = SolveOpts()
    lib.l1ls_solve_opts_default(ctypes.byref(o))
    names = {"tol": "rel_gap_tol"}
    for k, v in kw.items():
        k = names.get(k, k)
        if not hasattr(o, k):
            raise TypeError("unknown solver option %s" % k)
        setattr(o, k, v)
    return o


class Context:
    """An l1ls context on one CUDA device."""

    def __init__(self, device=0, budget_bytes=0):
        h = _P()
        _check(lib.l1ls_create(int(device), int(budget_bytes), ctypes.byref(h)))
        self._h = h
        self.device = device

    def generate(self, params, stream=None):
        p = gen_params(params) if isinstance(params, dict) else params
        h = _P()
        _check(lib.l1ls_generate(self._h, ctypes.byref(p), _stream_ptr(stream), ctypes.byref(h)))
        return Instance(self, h)

    # ---- serving ----------------------------------------------------------------------
    def serve_config(self, slots=8, capacity_bytes=0):
        _check(lib.l1ls_serve_config(self._h, int(slots), int(capacity_bytes)))

    def submit(self, params, method="fista", **opts):
        """Queue a solve request (generate + solve); returns its ticket."""
        p = gen_params(params) if isinstance(params, dict) else params
        o = solve_opts(**opts)
        t = ctypes.c_uint64()
        _check(lib.l1ls_submit(self._h, ctypes.byref(p), ctypes.byref(o), METHODS.get(method, method), ctypes.byref(t)))
        return t.value

    def poll(self, ticket, wait_ms=0, n=None):
        """None while the request runs; else (status, result dict, x or None)."""
        res = Result()
        x = np.zeros(n) if n else None
        st = lib.l1ls_poll(self._h, ctypes.c_uint64(ticket), int(wait_ms), ctypes.byref(res),
                           x.ctypes.data_as(_P) if x is not None else None)
        if st == 7:          # EBUSY: not finished
            return None
        if st == 8:
            _check(st)
        return st, res.as_dict(), x

    def cancel(self, ticket):
        _check(lib.l1ls_cancel(self._h, ctypes.c_uint64(ticket)))

    def serve_stats(self):
        i = ServeInfo()
        _check(lib.l1ls_serve_stats(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in ServeInfo._fields_ if k != "reserved0"}

    def close(self):
        if self._h:
            _check(lib.l1ls_destroy(self._h))
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Instance:
    """A generated instance resident on the device (row order of all m-vectors: original)."""

    def __init__(self, ctx, h):
        self.ctx = ctx
        self._h = h
        info = InstInfo()
        _check(lib.l1ls_inst_get_info(h, ctypes.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in InstInfo._fields_}
        self.m, self.n, self.nnz = info.m, info.n, info.nnz

    def refresh_info(self):
        """Re-read the instance info (device_bytes grows when solver work spaces are allocated)."""
        info = InstInfo()
        _check(lib.l1ls_inst_get_info(self._h, ctypes.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in InstInfo._fields_}
        return self.info

    def free(self):
        if self._h:
            _check(lib.l1ls_inst_free(self._h))
            self._h = None

    def export(self):
        m, n, nnz = self.m, self.n, self.nnz
        rp = np.zeros(m + 1, np.int64)
        ci = np.zeros(nnz, np.int32)
        va = np.zeros(nnz, np.float64)
        b = np.zeros(m, np.float64)
        xs = np.zeros(n, np.float64)
        sg = np.zeros(min(m, n), np.float64)
        pm = np.zeros(m, np.int64)
        _check(lib.l1ls_inst_export(self._h, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, b.ctypes.data,
                                    xs.ctypes.data, sg.ctypes.data, pm.ctypes.data))
        return dict(indptr=rp, indices=ci, data=va, b=b, xstar=xs, sigma=sg, perm=pm)

    def export_vectors(self):
        """b (original row order), x*, sigma and the row permutation, without the matrix."""
        m, n = self.m, self.n
        b = np.zeros(m, np.float64)
        xs = np.zeros(n, np.float64)
        sg = np.zeros(min(m, n), np.float64)
        pm = np.zeros(m, np.int64)
        _check(lib.l1ls_inst_export(self._h, None, None, None, b.ctypes.data, xs.ctypes.data, sg.ctypes.data,
                                    pm.ctypes.data))
        return dict(b=b, xstar=xs, sigma=sg, perm=pm)

    def xstar(self):
        """The generator's optimal x* (n doubles) without exporting the matrix."""
        xs = np.zeros(self.n, np.float64)
        _check(lib.l1ls_inst_export(self._h, None, None, None, None, xs.ctypes.data, None, None))
        return xs

    def kappa_rho(self, rho):
        """kappa_rho(x*) of Eq. (bd12), computed on the device (IGen instances)."""
        out = ctypes.c_double(0.0)
        _check(lib.l1ls_inst_kappa_rho(self._h, float(rho), ctypes.byref(out)))
        return out.value

    def export_t(self):
        cp = np.zeros(self.n + 1, np.int64)
        ri = np.zeros(self.nnz, np.int32)
        va = np.zeros(self.nnz, np.float64)
        _check(lib.l1ls_inst_export_t(self._h, cp.ctypes.data, ri.ctypes.data, va.ctypes.data))
        return dict(indptr=cp, indices=ri, data=va)

    def _product(self, fn, vin, vout, nin, nout, stream, device_only=False):
        if device_only:
            for v in (vin, vout):
                if not (hasattr(v, "is_cuda") and v.is_cuda):
                    raise ValueError("this product takes CUDA tensors for its input and output")
        if _numel(vin) != nin:
            raise ValueError("input vector has %d entries, the product needs %d" % (_numel(vin), nin))
        if vout is not None and _numel(vout) != nout:
            raise ValueError("output vector has %d entries, the product writes %d" % (_numel(vout), nout))
        pin, code, keep_in = _vec_ptr(vin)
        if vout is None:
            try:
                import torch
                if isinstance(vin, torch.Tensor):
                    vout = torch.empty(nout, dtype=vin.dtype, device=vin.device)
            except ImportError:
                pass
            if vout is None:
                vout = np.empty(nout, dtype=np.float64 if code == F64 else np.float32)
        pout, code_out, keep_out = _vec_ptr(vout)
        if code_out != code:
            raise ValueError("input and output vectors must have the same dtype")
        _check(fn(self._h, pin, code, pout, _stream_ptr(stream)))
        return vout

    def matvec(self, x, y=None, stream=None):
        """y = A x."""
        return self._product(lib.l1ls_matvec, x, y, self.n, self.m, stream)

    def rmatvec(self, y, x=None, stream=None):
        """x = A^T y."""
        return self._product(lib.l1ls_rmatvec, y, x, self.m, self.n, stream)

    def rmatvec_noalloc(self, y, x, stream=None):
        """x = A^T y with CUDA tensors and no allocation (fixed scratch, m <= 2^20)."""
        return self._product(lib.l1ls_rmatvec_noalloc, y, x, self.m, self.n, stream, device_only=True)

    def _solve(self, fn, x0, x_out, stream, opts, allow):
        o = opts if isinstance(opts, SolveOpts) else solve_opts(**opts)
        p0 = _vec_ptr(x0)[0] if x0 is not None else None
        keep0 = x0
        if x_out is None:
            x_out = np.zeros(self.n, np.float64)
        pout = _vec_ptr(x_out)[0]
        res = Result()
        st = fn(self._h, ctypes.byref(o), p0, pout, ctypes.byref(res), _stream_ptr(stream))
        del keep0
        _check(st, allow=allow)
        return x_out, res.as_dict()

    def solve_fista(self, x0=None, x_out=None, stream=None, allow=(4, 5), **opts):
        """FISTA to the duality-gap tolerance; returns (x, result dict)."""
        return self._solve(lib.l1ls_solve_fista, x0, x_out, stream, opts, allow)

    def solve_fista_bt(self, L0, eta=2.0, x0=None, x_out=None, stream=None, allow=(4, 5), **opts):
        """FISTA with backtracking on L from L0 (factor eta); returns (x, result dict)."""
        fn = lambda h, o, p0, pout, r, s: lib.l1ls_solve_fista_bt(h, o, float(L0), float(eta), p0, pout, r, s)
        return self._solve(fn, x0, x_out, stream, opts, allow)

    def fista_begin(self, x0=None, stream=None, **opts):
        o = solve_opts(**opts)
        p0 = _vec_ptr(x0)[0] if x0 is not None else None
        _check(lib.l1ls_fista_begin(self._h, ctypes.byref(o), p0, _stream_ptr(stream)))

    def fista_step(self, iters=1, timed=False, stream=None):
        """Enqueue iterations; with timed=True returns the summed K1 / K2 times in ms."""
        ms = (ctypes.c_float * 2)()
        _check(lib.l1ls_fista_step(self._h, int(iters), ms if timed else None, _stream_ptr(stream)))
        return (ms[0], ms[1]) if timed else None

    def fista_end(self, x_out=None, stream=None, allow=(4, 5)):
        res = Result()
        pout = _vec_ptr(x_out)[0] if x_out is not None else None
        _check(lib.l1ls_fista_end(self._h, pout, ctypes.byref(res), _stream_ptr(stream)), allow=allow)
        return x_out, res.as_dict()

    def solve_pdncg(self, x0=None, x_out=None, stream=None, allow=(4, 5), **opts):
        """Primal-dual Newton-CG to the duality-gap tolerance; returns (x, result dict)."""
        return self._solve(lib.l1ls_solve_pdncg, x0, x_out, stream, opts, allow)


class Batch:
    """A ragged batch of instances (paired storage, FP32 or BF16 values) solved together."""

    def __init__(self, ctx, instances):
        self.ctx = ctx
        self.instances = list(instances)
        arr = (_P * len(self.instances))(*[i._h for i in self.instances])
        h = _P()
        _check(lib.l1ls_batch_create(ctx._h, len(self.instances), arr, ctypes.byref(h)))
        self._h = h

    def solve_path(self, taus, x_out=None, stream=None, allow=(4, 5), **opts):
        """taus: (count, ntau) array.  Returns a list (per instance) of lists (per tau) of result dicts."""
        t = np.ascontiguousarray(np.asarray(taus, dtype=np.float64))
        count, ntau = t.shape
        o = solve_opts(**opts)
        res = (Result * (count * ntau))()
        xs = None
        keep = []
        if x_out is not None:
            ptrs = []
            for v in x_out:
                if v is None:
                    ptrs.append(None)
                else:
                    p, _, k = _vec_ptr(v)
                    keep.append(k)
                    ptrs.append(p.value)
            xs = (_P * count)(*ptrs)
        st = lib.l1ls_batch_solve_path(self._h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ntau,
                                       ctypes.byref(o), res, xs, _stream_ptr(stream))
        _check(st, allow=allow)
        return [[res[i * ntau + j].as_dict() for j in range(ntau)] for i in range(count)]

    def schedule(self):
        """The autotuned schedule: block size, entries per lane, probe times of the 4 candidates."""
        b = ctypes.c_int()
        e = ctypes.c_int()
        ms = (ctypes.c_double * 4)()
        _check(lib.l1ls_batch_get_schedule(self._h, ctypes.byref(b), ctypes.byref(e), ms))
        return {"block": b.value, "entries_per_lane": e.value, "probe_ms": list(ms),
                "candidates": [(256, 0), (128, 0), (256, 8), (128, 8)]}

    def barrier_selftest(self, max_polls=1 << 12):
        """Run the bounded-barrier self-test; returns (status, message, seconds)."""
        sec = ctypes.c_double()
        st = lib.l1ls_batch_barrier_selftest(self._h, int(max_polls), ctypes.byref(sec))
        return st, lib.l1ls_last_error().decode(), sec.value

    def stats(self):
        """Of the last solve: batch steps run and the device time of their launches (ms)."""
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(lib.l1ls_batch_get_stats(self._h, ctypes.byref(n), ctypes.byref(ms)))
        return {"steps": n.value, "device_ms": ms.value}

    def free(self):
        if self._h:
            _check(lib.l1ls_batch_free(self._h))
            self._h = None


def footprint(params, method="fista"):
    """Device bytes the serving loop reserves for a request (an upper bound)."""
    p = gen_params(params) if isinstance(params, dict) else params
    return lib.l1ls_footprint(ctypes.byref(p), METHODS.get(method, method))


def version():
    return lib.l1ls_version().decode()
