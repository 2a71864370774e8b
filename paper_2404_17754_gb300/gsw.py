"""Python binding of the GPU library's C ABI (``include/gsw.h``).

Argument marshalling only: every step of the analysis runs in the library's
CUDA kernels.  PyTorch supplies device memory (its caching allocator backs
the library's allocations) and the CUDA stream.  The library must be built
(``paper_2404_17754_gb300.build.build()``); importing this module without it
raises, and there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsw.so")

OK, E_INVALID, E_CUDA, E_NOMEM, E_NOCONV, E_NAN, E_TIMEOUT, E_STATE = 0, -1, -2, -3, -4, -5, -6, -7
PREC_FP64, PREC_FP32, PREC_FP16 = 0, 1, 2
OUTER_AUTO, OUTER_FP64, OUTER_DWORD = 0, 1, 2
_STATUS = {E_INVALID: "GSW_E_INVALID", E_CUDA: "GSW_E_CUDA", E_NOMEM: "GSW_E_NOMEM",
           E_NOCONV: "GSW_E_NOCONV", E_NAN: "GSW_E_NAN", E_TIMEOUT: "GSW_E_TIMEOUT",
           E_STATE: "GSW_E_STATE"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)
_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class SolverOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("inner_iters", C.c_int32), ("check_every", C.c_int32), ("batch_outer", C.c_int32),
                ("inner_variant", C.c_int32), ("inner_rtol", C.c_double), ("guess_order", C.c_int32),
                ("outer_op", C.c_int32), ("share_dirs", C.c_int32), ("proj_dim", C.c_int32),
                ("coarse_weight", C.c_double), ("coarse_relres", C.c_double), ("proj_relres", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("steps_done", C.c_int64), ("cg_iters_total", C.c_int64), ("cg_iters_last", C.c_int32),
                ("cg_iters_max", C.c_int32), ("relres_last", C.c_double), ("inner_iters_total", C.c_int64),
                ("kernel_launches", C.c_int64), ("init_relres_sum", C.c_double)]


class LearnOpts(C.Structure):
    _fields_ = [("enable", C.c_int32), ("train_steps", C.c_int32), ("batch", C.c_int32),
                ("iters_per_step", C.c_int32), ("lr", C.c_float), ("seed", C.c_uint32)]


_fp = C.POINTER(C.c_float)


class GswError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


_lib = None

# entry point -> (restype, argtypes)
SIGNATURES = {
    "gsw_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "gsw_destroy": (None, [C.c_void_p]),
    "gsw_last_error": (C.c_char_p, [C.c_void_p]),
    "gsw_set_allocator": (C.c_int, [C.c_void_p, _ALLOC, _FREE, C.c_void_p]),
    "gsw_model_upload": (C.c_int, [C.c_void_p, C.c_int64, _dp, C.c_int64, _ip, _ip, C.c_int32, _dp,
                                   C.c_int64, _ip, _ip, _ip, _dp, C.c_int32, _dp, _ip]),
    "gsw_model_free": (C.c_int, [C.c_void_p, C.c_int32]),
    "gsw_model_info": (C.c_int, [C.c_void_p, C.c_int32, _lp]),
    "gsw_set_time": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.c_double, C.c_double]),
    "gsw_set_input": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, _dp, C.c_int32]),
    "gsw_set_solver": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(SolverOpts)]),
    "gsw_reset": (C.c_int, [C.c_void_p, C.c_int32]),
    "gsw_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "gsw_run": (C.c_int, [C.c_void_p, _ip, C.c_int32, C.c_int32]),
    "gsw_batch_create": (C.c_int, [C.c_void_p, _ip, C.c_int32, _ip]),
    "gsw_batch_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "gsw_batch_destroy": (C.c_int, [C.c_void_p, C.c_int32]),
    "gsw_batch_launches": (C.c_int, [C.c_void_p, C.c_int32, _lp]),
    "gsw_read_waveforms": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, _dp]),
    "gsw_read_waveform_steps": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, _dp]),
    "gsw_timing": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, _dp, _lp]),
    "gsw_stats_get": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(Stats)]),
    "gsw_checkpoint": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_size_t)]),
    "gsw_restore": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t]),
    "gsw_get_state": (C.c_int, [C.c_void_p, C.c_int32, _dp, _dp, _dp, _lp]),
    "gsw_set_state": (C.c_int, [C.c_void_p, C.c_int32, _dp, _dp, _dp, C.c_int64]),
    "gsw_apply": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "gsw_read_preconditioner": (C.c_int, [C.c_void_p, C.c_int32, _dp]),
    "gsw_read_receivers": (C.c_int, [C.c_void_p, C.c_int32, _ip, _dp]),
    "gsw_wait_probe": (C.c_int, [C.c_void_p, C.c_int64]),
    "gsw_misfit": (C.c_int, [C.c_void_p, C.c_int32, _dp, C.c_int32, C.c_int32, C.c_double, _dp, _dp]),
    "gsw_misfit_green": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, _dp, _dp, C.c_int32, C.c_int32, C.c_double,
                                   _dp, _dp]),
    "gsw_set_learning": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(LearnOpts)]),
    "gsw_mlp_train": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(LearnOpts)]),
    "gsw_mlp_params": (C.c_int, [C.c_void_p, C.c_int32, _dp, _dp]),
    "gsw_mlp_forward": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "gsw_mlp_grad": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, _dp, _dp]),
    "gsw_mlp_state": (C.c_int, [C.c_void_p, C.c_int32, _dp]),
    "gsw_mlp_inputs": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, _ip, C.c_void_p, _dp,
                                 _dp]),
    "gsw_misfit_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                     C.c_int32, C.c_double, C.c_void_p, C.c_void_p]),
}


def load(path=LIB_PATH):
    """Load libgsw.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libgsw.so is not built (%s); run paper_2404_17754_gb300.build.build()" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


class Context:
    """A library context bound to one GPU and one CUDA stream.

    ``stream``: a ``torch.cuda.Stream`` (default: torch's current stream on
    ``device``).  ``torch_alloc``: back device allocations by torch's caching
    allocator.
    """

    def __init__(self, device=0, stream=None, torch_alloc=True):
        import torch

        self.lib = load()
        self.device = device
        self._torch = torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        st = self.lib.gsw_create(C.byref(h), device, C.c_void_p(stream.cuda_stream))
        if st != OK:
            raise GswError(st, "gsw_create(device=%d)" % device)
        self.h = h
        self._cbs = None
        if torch_alloc:
            dev = device

            def _alloc(nbytes, strm, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm)
                except Exception:  # out of memory: report NULL to the library
                    return None

            def _free(ptr, strm, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cbs = (_ALLOC(_alloc), _FREE(_free))
            self._check(self.lib.gsw_set_allocator(self.h, self._cbs[0], self._cbs[1], None))

    def _check(self, st):
        if st != OK:
            raise GswError(st, self.lib.gsw_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.gsw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload(self, mesh, mat, rec_xy):
        """Upload a mesh dict (``synth.mesh.layered_box`` layout); returns a :class:`Model`."""
        xyz, pxyz = _d(mesh["xyz"])
        conn, pconn = _i(mesh["conn"])
        em, pem = _i(mesh["elem_mat"])
        mt, pmt = _d(mat)
        fc, pfc = _i(mesh["faces"])
        fe, pfe = _i(mesh["face_elem"])
        ft, pft = _i(mesh["face_tag"])
        per, pper = _d(mesh.get("period", np.zeros(2)))
        rc, prc = _d(np.asarray(rec_xy, dtype=np.float64).reshape(-1, 2))
        mid = C.c_int32()
        self._check(self.lib.gsw_model_upload(self.h, xyz.shape[0], pxyz, conn.shape[0], pconn, pem, mt.shape[0],
                                              pmt, fc.shape[0], pfc, pfe, pft, pper, rc.shape[0], prc,
                                              C.byref(mid)))
        return Model(self, mid.value, xyz.shape[0], rc.shape[0])

    def misfit_green(self, G, obs, stride, n_shifts, tau=1e-10):
        """(ERR, c [3, n_shifts]) of Eq. (2) for Green's functions G [n_rec, 3, 3, n_t] given on the host
        and observations obs [n_rec, 3, n_t]."""
        G, pG = _d(G)
        obs, pO = _d(obs)
        n_rec, n_t = obs.shape[0], obs.shape[2]
        assert G.shape == (n_rec, 3, 3, n_t)
        err = C.c_double()
        c = np.zeros((3, n_shifts))
        self._check(self.lib.gsw_misfit_green(self.h, n_rec, n_t, pG, pO, stride, n_shifts, tau, C.byref(err),
                                              c.ctypes.data_as(_dp)))
        return err.value, c

    def wait_probe(self, limit):
        """Failure-detection self-test: the bounded device-side wait on a barrier nothing completes.
        Returns the library status (``E_TIMEOUT`` expected) without raising."""
        return int(self.lib.gsw_wait_probe(self.h, int(limit)))

    def run(self, models, dirs_mask=0):
        """Run analyses from rest to the end, batched: each model's own analysis (dirs_mask 0) or, for
        every model, the analysis of each input direction in dirs_mask (bits x1, x2, x3)."""
        ids = np.array([m.id for m in models], dtype=np.int32)
        self._check(self.lib.gsw_run(self.h, ids.ctypes.data_as(_ip), len(ids), int(dirs_mask)))


    def misfit_noalloc(self, G_dev, obs_dev, stride, n_shifts, err_dev, c_dev=None, tau=1e-10):
        """Allocation-free misfit on caller-owned CUDA float64 tensors.

        For callers that cannot allocate device memory: G_dev [n_rec, 3, 3, n_t],
        obs_dev [n_rec, 3, n_t] are inputs, err_dev (1 element) and c_dev
        [3, n_shifts] (optional) receive the results.  Nothing is allocated; the
        work is queued on the context's stream.  Limits: n_shifts <= 64, n_rec <= 1024.
        """
        for t in (G_dev, obs_dev, err_dev) + ((c_dev,) if c_dev is not None else ()):
            if not (t.is_cuda and t.is_contiguous() and t.dtype == self._torch.float64):
                raise ValueError("device arguments must be contiguous CUDA float64 tensors")
        if obs_dev.dim() != 3 or obs_dev.shape[1] != 3:
            raise ValueError("obs_dev must have shape (n_rec, 3, n_t)")
        n_rec, n_t = obs_dev.shape[0], obs_dev.shape[2]
        if tuple(G_dev.shape) != (n_rec, 3, 3, n_t):
            raise ValueError("G_dev must have shape (n_rec, 3, 3, n_t) = (%d, 3, 3, %d)" % (n_rec, n_t))
        if err_dev.numel() < 1:
            raise ValueError("err_dev must hold at least one element")
        if c_dev is not None and c_dev.numel() != 3 * n_shifts:
            raise ValueError("c_dev must hold 3 * n_shifts = %d elements" % (3 * n_shifts))
        self._check(self.lib.gsw_misfit_noalloc(self.h, n_rec, n_t, C.c_void_p(G_dev.data_ptr()),
                                                C.c_void_p(obs_dev.data_ptr()), stride, n_shifts, tau,
                                                C.c_void_p(err_dev.data_ptr()),
                                                C.c_void_p(c_dev.data_ptr() if c_dev is not None else 0)))


    def batch(self, models):
        """Group models (mixed precision) for batched, graph-captured stepping."""
        return Batch(self, models)


class Batch:
    """Models advanced together, one captured CUDA graph launch per time step."""

    def __init__(self, ctx, models):
        self.ctx = ctx
        self.models = list(models)
        ids = np.array([m.id for m in self.models], dtype=np.int32)
        bid = C.c_int32()
        ctx._check(ctx.lib.gsw_batch_create(ctx.h, ids.ctypes.data_as(_ip), len(ids), C.byref(bid)))
        self.id = bid.value

    def step(self, n=1):
        self.ctx._check(self.ctx.lib.gsw_batch_step(self.ctx.h, self.id, int(n)))

    def launches_per_step(self):
        n = C.c_int64()
        self.ctx._check(self.ctx.lib.gsw_batch_launches(self.ctx.h, self.id, C.byref(n)))
        return n.value

    def close(self):
        if self.id:
            self.ctx._check(self.ctx.lib.gsw_batch_destroy(self.ctx.h, self.id))
            self.id = 0


class Model:
    """One uploaded ground model (handle into a :class:`Context`)."""

    def __init__(self, ctx, mid, n_nodes, n_rec):
        self.ctx, self.id, self.n_nodes, self.n_rec = ctx, mid, n_nodes, n_rec
        self.n_steps = 0

    def _c(self, st):
        self.ctx._check(st)

    def info(self):
        out = np.zeros(6, dtype=np.int64)
        self._c(self.ctx.lib.gsw_model_info(self.ctx.h, self.id, out.ctypes.data_as(_lp)))
        return dict(n_nodes=int(out[0]), n_elem=int(out[1]), n_faces=int(out[2]), n_rec=int(out[3]),
                    device_bytes=int(out[4]), inner_variant=int(out[5]))

    def set_time(self, dt, n_steps, band):
        self._c(self.ctx.lib.gsw_set_time(self.ctx.h, self.id, float(dt), int(n_steps), float(band[0]),
                                          float(band[1])))
        self.n_steps = int(n_steps)

    def set_input(self, direction, p):
        p, pp = _d(p)
        self._c(self.ctx.lib.gsw_set_input(self.ctx.h, self.id, int(direction), pp, p.shape[0]))

    def set_solver(self, tol=1e-8, max_iter=10000, precision=PREC_FP64, inner_iters=20, check_every=8,
                   batch_outer=6, inner_variant=-1, inner_rtol=0.0, guess_order=0, outer_op=OUTER_AUTO,
                   share_dirs=0, proj_dim=0, coarse_weight=0.0, coarse_relres=0.0, proj_relres=0.0):
        o = SolverOpts(tol, max_iter, precision, inner_iters, check_every, batch_outer, inner_variant, inner_rtol,
                       guess_order, outer_op, int(share_dirs), int(proj_dim), float(coarse_weight),
                       float(coarse_relres), float(proj_relres))
        self._c(self.ctx.lib.gsw_set_solver(self.ctx.h, self.id, C.byref(o)))

    def reset(self):
        self._c(self.ctx.lib.gsw_reset(self.ctx.h, self.id))

    def step(self, n=1):
        self._c(self.ctx.lib.gsw_step(self.ctx.h, self.id, int(n)))

    def run(self, dirs_mask=0):
        ids = np.array([self.id], dtype=np.int32)
        self._c(self.ctx.lib.gsw_run(self.ctx.h, ids.ctypes.data_as(_ip), 1, int(dirs_mask)))

    def waveforms(self, direction=-1):
        """Receiver history [n_rec, 3, n_steps] of the model's own analysis (-1) or of the analysis of input
        direction 0..2 run by ``run(dirs_mask)``."""
        out = np.zeros((self.n_rec, 3, self.n_steps))
        self._c(self.ctx.lib.gsw_read_waveforms(self.ctx.h, self.id, int(direction), out.ctypes.data_as(_dp)))
        return out

    def read_waveforms_into(self, out, direction=-1):
        """Read the receiver history into a caller-owned float64 host array."""
        self._c(self.ctx.lib.gsw_read_waveforms(self.ctx.h, self.id, int(direction), out.ctypes.data_as(_dp)))
        return out

    def misfit(self, obs, stride, n_shifts, tau=1e-10):
        """(ERR, c [3, n_shifts]) of Eq. (2) against observations obs [n_rec, 3, n_steps], from the model's
        three input-direction analyses (``run(dirs_mask=7)``), computed on the device."""
        obs, pO = _d(obs)
        err = C.c_double()
        c = np.zeros((3, n_shifts))
        self._c(self.ctx.lib.gsw_misfit(self.ctx.h, self.id, pO, int(stride), int(n_shifts), float(tau),
                                        C.byref(err), c.ctypes.data_as(_dp)))
        return err.value, c

    def checkpoint(self):
        """Full checkpoint (state, receiver history, increment history, learned-guess state) as bytes."""
        n = C.c_size_t(0)
        self._c(self.ctx.lib.gsw_checkpoint(self.ctx.h, self.id, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._c(self.ctx.lib.gsw_checkpoint(self.ctx.h, self.id, buf, C.byref(n)))
        return buf.raw

    def restore(self, data):
        buf = C.create_string_buffer(bytes(data), len(data))
        self._c(self.ctx.lib.gsw_restore(self.ctx.h, self.id, buf, len(data)))

    def read_steps_into(self, step0, out):
        """Receiver velocities of steps step0 .. step0 + out.shape[2] - 1 into a host array."""
        self._c(self.ctx.lib.gsw_read_waveform_steps(self.ctx.h, self.id, int(step0), int(out.shape[2]),
                                                     out.ctypes.data_as(_dp)))
        return out

    def timing(self, enable=None):
        """Start (True) / stop (False) / query (None) operator launch timing.

        Returns {"fp64": (ms, launches), "inner": (ms, launches)}.
        """
        ms = np.zeros(2)
        n = np.zeros(2, dtype=np.int64)
        flag = -1 if enable is None else int(bool(enable))
        self._c(self.ctx.lib.gsw_timing(self.ctx.h, self.id, flag, ms.ctypes.data_as(_dp), n.ctypes.data_as(_lp)))
        return {"fp64": (float(ms[0]), int(n[0])), "inner": (float(ms[1]), int(n[1]))}

    def stats(self, direction=-1):
        s = Stats()
        self._c(self.ctx.lib.gsw_stats_get(self.ctx.h, self.id, int(direction), C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def get_state(self):
        u, v, a = (np.zeros((self.n_nodes, 3)) for _ in range(3))
        step = C.c_int64()
        self._c(self.ctx.lib.gsw_get_state(self.ctx.h, self.id, u.ctypes.data_as(_dp), v.ctypes.data_as(_dp),
                                           a.ctypes.data_as(_dp), C.byref(step)))
        return u, v, a, step.value

    def set_state(self, u, v, a, step):
        u, pu = _d(u)
        v, pv = _d(v)
        a, pa = _d(a)
        self._c(self.ctx.lib.gsw_set_state(self.ctx.h, self.id, pu, pv, pa, int(step)))

    def apply(self, which, x):
        """y = A x (0), K x (1), M x (2), C x (3), A x by the inner reduced-precision operator (4), A x
        in double-word arithmetic (5), or the two-level inner preconditioner's coarse correction
        P D_c^-1 P^T x (6)."""
        torch = self.ctx._torch
        assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous() and x.numel() == 3 * self.n_nodes
        y = torch.empty_like(x)
        self._c(self.ctx.lib.gsw_apply(self.ctx.h, self.id, int(which), C.c_void_p(x.data_ptr()),
                                       C.c_void_p(y.data_ptr())))
        return y

    def preconditioner(self):
        out = np.zeros((self.n_nodes, 6))
        self._c(self.ctx.lib.gsw_read_preconditioner(self.ctx.h, self.id, out.ctypes.data_as(_dp)))
        return out

    def receivers(self):
        nodes = np.zeros((self.n_rec, 6), dtype=np.int32)
        w = np.zeros((self.n_rec, 6))
        self._c(self.ctx.lib.gsw_read_receivers(self.ctx.h, self.id, nodes.ctypes.data_as(_ip),
                                                w.ctypes.data_as(_dp)))
        return nodes, w

    def set_learning(self, enable=True, train_steps=500, batch=16384, iters_per_step=2, lr=1e-3, seed=1):
        o = LearnOpts(int(enable), int(train_steps), int(batch), int(iters_per_step), float(lr), int(seed))
        self._c(self.ctx.lib.gsw_set_learning(self.ctx.h, self.id, C.byref(o)))

    def mlp_train(self, n_train_steps, batch=16384, iters_per_step=2, lr=1e-3, seed=1):
        """Train the learned guess on the next n_train_steps steps (advancing them); later steps apply it."""
        o = LearnOpts(1, 0, int(batch), int(iters_per_step), float(lr), int(seed))
        self._c(self.ctx.lib.gsw_mlp_train(self.ctx.h, self.id, int(n_train_steps), C.byref(o)))

    def mlp_params(self, set_to=None):
        out = np.zeros(5443)
        src = None
        if set_to is not None:
            src = np.ascontiguousarray(set_to, dtype=np.float64)
        self._c(self.ctx.lib.gsw_mlp_params(self.ctx.h, self.id, out.ctypes.data_as(_dp),
                                            src.ctypes.data_as(_dp) if src is not None else None))
        return out

    def mlp_forward(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        out = np.zeros((X.shape[0], 3), dtype=np.float32)
        self._c(self.ctx.lib.gsw_mlp_forward(self.ctx.h, self.id, X.shape[0], X.ctypes.data, out.ctypes.data))
        return out

    def mlp_grad(self, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        loss = C.c_double()
        g = np.zeros(5443)
        self._c(self.ctx.lib.gsw_mlp_grad(self.ctx.h, self.id, X.shape[0], X.ctypes.data, Y.ctypes.data,
                                          C.byref(loss), g.ctypes.data_as(_dp)))
        return loss.value, g

    def mlp_state(self):
        out = np.zeros(5)
        self._c(self.ctx.lib.gsw_mlp_state(self.ctx.h, self.id, out.ctypes.data_as(_dp)))
        return dict(loss=out[0], active=bool(out[1]), plain_r0=out[2], learned_r0=out[3], learned_steps=int(out[4]))

    def mlp_inputs(self, nodes, batch):
        """The last training batch (X [batch, 16], Y [batch, 3]) and, for ``nodes``, the
        features [n, 16], base guess [n, 3] and (sigma, output scale) of the next step."""
        nodes, pn = _i(nodes)
        n = nodes.shape[0]
        Xt = np.zeros((batch, 16), dtype=np.float32)
        Yt = np.zeros((batch, 3), dtype=np.float32)
        X = np.zeros((max(n, 1), 16), dtype=np.float32)
        base = np.zeros((max(n, 1), 3))
        scale = np.zeros(2)
        self._c(self.ctx.lib.gsw_mlp_inputs(self.ctx.h, self.id, Xt.ctypes.data, Yt.ctypes.data, n, pn,
                                            X.ctypes.data, base.ctypes.data_as(_dp), scale.ctypes.data_as(_dp)))
        return dict(x_train=Xt, y_train=Yt, x=X[:n], base=base[:n], sigma=scale[0], scale=scale[1])

    def mlp_loss(self):
        return self.mlp_state()["loss"]

    def free(self):
        self._c(self.ctx.lib.gsw_model_free(self.ctx.h, self.id))


def analysis(ctx, cfg, tol=1e-8, n_steps=None, **solver):
    """Upload a ``synth.configs`` workload, run it, return (waveforms, stats, model)."""
    n = cfg["n_steps"] if n_steps is None else n_steps
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], n, cfg["band"])
    m.set_input(cfg["dir"], np.asarray(cfg["p"][:n]))
    m.set_solver(tol=tol, **solver)
    m.run()
    return m.waveforms(), m.stats(), m
