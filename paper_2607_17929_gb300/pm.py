"""Python binding of libpm's C ABI (include/pm.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays may
be torch tensors (CUDA or CPU) or numpy arrays; the library itself decides
whether a pointer is host or device memory.  There is no fallback: if
libpm.so is missing the import fails with instructions.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libpm.so")

PM_OK, PM_ERR_INVALID_ARG, PM_ERR_UNSUPPORTED_SIZE, PM_ERR_OOM, PM_ERR_CUDA, PM_ERR_TIMEOUT, PM_ERR_STATE = range(7)
STATUS_NAMES = {0: "PM_OK", 1: "PM_ERR_INVALID_ARG", 2: "PM_ERR_UNSUPPORTED_SIZE", 3: "PM_ERR_OOM",
                4: "PM_ERR_CUDA", 5: "PM_ERR_TIMEOUT", 6: "PM_ERR_STATE"}
PM_FP64, PM_MIXED = 0, 1
PM_NEWTONIAN, PM_FULL_HC, PM_B_SPACESPACE = 1, 2, 4
FIELDS = {"phi": 0, "chi": 1, "Bx": 2, "By": 3, "Bz": 4, "R": 5, "Fx": 6, "Fy": 7, "Fz": 8,
          "Sxx": 9, "Sxy": 10, "Sxz": 11, "Syy": 12, "Syz": 13}
TENSORS = {"h+": 0, "hx": 1, "h+'": 2, "hx'": 3}
TIMINGS = ["project", "fft_fwd", "solve", "fft_inv", "kick_drift", "sort", "step", "fft_fwd_x", "fft_fwd_y",
           "fft_fwd_z", "fft_inv_z", "fft_inv_y", "fft_inv_x", "scan", "scatter"]


class pm_config(C.Structure):
    _fields_ = [("n_mesh", C.c_int32), ("n_steps", C.c_int32), ("n_part", C.c_int64),
                ("box_mpch", C.c_double), ("omega_m", C.c_double), ("z_init", C.c_double),
                ("z_final", C.c_double), ("precision", C.c_int32), ("flags", C.c_uint32),
                ("stream", C.c_void_p)]


class PMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(_SO):
        raise ImportError(f"{_SO} is missing: build it with `python -m paper_2607_17929_gb300.build` "
                          "(nvcc, sm_103a); there is no CPU fallback")
    L = C.CDLL(_SO)
    vp, dp, i32, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int64
    sig = {
        "pm_init": ([C.POINTER(pm_config), C.POINTER(vp)], C.c_int),
        "pm_destroy": ([vp], None),
        "pm_last_error": ([vp], C.c_char_p),
        "pm_set_particles": ([vp, vp, vp], C.c_int),
        "pm_project": ([vp], C.c_int),
        "pm_solve": ([vp], C.c_int),
        "pm_update": ([vp], C.c_int),
        "pm_step": ([vp], C.c_int),
        "pm_step_graph": ([vp, C.c_int32], C.c_int),
        "pm_get_particles": ([vp, vp, vp], C.c_int),
        "pm_get_field": ([vp, C.c_int, vp], C.c_int),
        "pm_get_tensor": ([vp, C.c_int, vp], C.c_int),
        "pm_power_spectrum": ([vp, C.c_int, dp, dp, C.POINTER(i64)], C.c_int),
        "pm_get_time": ([vp, C.POINTER(i32), dp, dp], C.c_int),
        "pm_get_schedule": ([vp, dp, dp, dp], C.c_int),
        "pm_get_timings": ([vp, dp, C.c_int, C.POINTER(i64)], C.c_int),
        "pm_fft_shapes": ([vp, i32, i32, C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "pm_deposit_shape": ([vp, i32, C.POINTER(i32)], C.c_int),
        "pm_set_particles_packed": ([vp, vp], C.c_int),
        "pm_put_particles_packed": ([vp, vp], C.c_int),
        "pm_get_particles_packed": ([vp, vp], C.c_int),
        "pm_put_particles_packed_async": ([vp, vp], C.c_int),
        "pm_get_particles_packed_async": ([vp, vp], C.c_int),
        "pm_io_wait": ([vp], C.c_int),
        "pm_ensemble_set_batched": ([vp, i32], C.c_int),
        "pm_ensemble_get_mode": ([vp, C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "pm_put_particles": ([vp, vp, vp], C.c_int),
        "pm_ensemble_init": ([C.c_void_p, i32, C.POINTER(vp)], C.c_int),
        "pm_ensemble_destroy": ([vp], None),
        "pm_ensemble_last_error": ([vp], C.c_char_p),
        "pm_ensemble_box": ([vp, i32, C.POINTER(vp)], C.c_int),
        "pm_ensemble_set_particles": ([vp, i32, vp, vp], C.c_int),
        "pm_ensemble_step": ([vp, i32], C.c_int),
        "pm_ensemble_sync": ([vp], C.c_int),
        "pm_ensemble_tune": ([vp, C.POINTER(i32)], C.c_int),
        "pm_ensemble_stream": ([vp, C.POINTER(vp)], C.c_int),
        "pm_ensemble_set_streams": ([vp, i32], C.c_int),
        "pm_power_spectrum_noalloc": ([vp, i64, i32, C.c_double, i32, dp, dp, C.POINTER(i64), vp], C.c_int),
        "pm_net_param_count": ([], i64),
        "pm_net_create": ([i32, C.c_uint64, vp, C.POINTER(vp)], C.c_int),
        "pm_net_destroy": ([vp], None),
        "pm_net_last_error": ([vp], C.c_char_p),
        "pm_net_set_params": ([vp, vp], C.c_int),
        "pm_net_get_params": ([vp, vp], C.c_int),
        "pm_net_buffer": ([vp, i32, C.POINTER(vp)], C.c_int),
        "pm_net_features": ([vp, vp], C.c_int),
        "pm_net_target": ([vp, vp, vp, vp], C.c_int),
        "pm_net_forward": ([vp], C.c_int),
        "pm_net_backward": ([vp, vp, dp], C.c_int),
        "pm_net_adam": ([vp, C.c_float], C.c_int),
        "pm_net_train_step": ([vp, vp, C.c_float, dp], C.c_int),
        "pm_net_apply": ([vp, vp], C.c_int),
        "pm_set_correction": ([vp, vp], C.c_int),
        "pm_net_set_scales": ([vp, C.c_double, C.c_double, C.c_double], C.c_int),
        "pm_conv3d_forward": ([i32, vp, vp, vp, i32, i32, vp, vp], C.c_int),
        "pm_conv3d_backward_weight": ([i32, vp, vp, vp, vp], C.c_int),
        "pm_conv3d_check": ([vp], C.c_int),
        "pm_save": ([vp, C.c_char_p], C.c_int),
        "pm_load": ([vp, C.c_char_p], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()

EXPORTED = ["pm_init", "pm_destroy", "pm_last_error", "pm_set_particles", "pm_project", "pm_solve",
            "pm_update", "pm_step", "pm_step_graph", "pm_put_particles", "pm_get_particles", "pm_get_field", "pm_get_tensor", "pm_power_spectrum",
            "pm_power_spectrum_noalloc", "pm_ensemble_init", "pm_ensemble_destroy", "pm_ensemble_last_error",
            "pm_ensemble_box", "pm_ensemble_set_particles", "pm_ensemble_step", "pm_ensemble_sync", "pm_ensemble_tune",
            "pm_ensemble_stream", "pm_ensemble_set_streams", "pm_net_param_count", "pm_net_create", "pm_net_destroy", "pm_net_last_error",
            "pm_net_set_params", "pm_net_get_params", "pm_net_buffer", "pm_net_features", "pm_net_target",
            "pm_net_forward", "pm_net_backward", "pm_net_adam", "pm_net_train_step", "pm_net_apply",
            "pm_set_correction", "pm_net_set_scales", "pm_conv3d_forward", "pm_conv3d_backward_weight", "pm_conv3d_check",
            "pm_get_time", "pm_get_schedule", "pm_get_timings", "pm_fft_shapes", "pm_deposit_shape", "pm_save",
            "pm_load", "pm_ensemble_set_batched", "pm_ensemble_get_mode", "pm_set_particles_packed",
            "pm_put_particles_packed", "pm_get_particles_packed", "pm_put_particles_packed_async",
            "pm_get_particles_packed_async", "pm_io_wait"]


def _ptr(a):
    """Raw data pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream):
    """Raw cudaStream_t of a torch.cuda.Stream, a raw handle, or None (default stream)."""
    return None if stream is None else getattr(stream, "cuda_stream", stream)


def _check(ctx, st):
    if st != PM_OK:
        msg = lib.pm_last_error(ctx).decode() if ctx else ""
        raise PMError(st, msg)


def pm_init(n_mesh, n_part, box_mpch, omega_m, z_init, z_final=0.0, n_steps=100, precision=PM_FP64, flags=0,
            stream=None):
    """Create a context; returns an opaque handle (int).  stream: a torch.cuda.Stream, raw handle or None."""
    cfg = pm_config(int(n_mesh), int(n_steps), int(n_part), float(box_mpch), float(omega_m), float(z_init),
                    float(z_final), int(precision), int(flags), None)
    if stream is not None:
        cfg.stream = getattr(stream, "cuda_stream", stream)
    h = C.c_void_p()
    st = lib.pm_init(C.byref(cfg), C.byref(h))
    if st != PM_OK:
        raise PMError(st, "pm_init rejected the configuration or could not allocate")
    return h.value


def pm_destroy(ctx):
    lib.pm_destroy(ctx)


def pm_last_error(ctx):
    return lib.pm_last_error(ctx).decode()


def pm_set_particles(ctx, pos, mom):
    _check(ctx, lib.pm_set_particles(ctx, _ptr(pos), _ptr(mom)))


def pm_project(ctx):
    _check(ctx, lib.pm_project(ctx))


def pm_solve(ctx):
    _check(ctx, lib.pm_solve(ctx))


def pm_update(ctx):
    _check(ctx, lib.pm_update(ctx))


def pm_step(ctx):
    _check(ctx, lib.pm_step(ctx))


def pm_step_graph(ctx, on):
    """pm_step as one captured CUDA graph per step (on=1) or as plain launches (on=0, the default)."""
    _check(ctx, lib.pm_step_graph(ctx, int(on)))


def pm_put_particles(ctx, pos, mom):
    _check(ctx, lib.pm_put_particles(ctx, _ptr(pos), _ptr(mom)))


def pm_get_particles(ctx, pos, mom):
    _check(ctx, lib.pm_get_particles(ctx, _ptr(pos), _ptr(mom)))


def pm_get_field(ctx, field, dst):
    fid = FIELDS[field] if isinstance(field, str) else int(field)
    _check(ctx, lib.pm_get_field(ctx, fid, _ptr(dst)))


def pm_get_tensor(ctx, which, dst):
    wid = TENSORS[which] if isinstance(which, str) else int(which)
    _check(ctx, lib.pm_get_tensor(ctx, wid, _ptr(dst)))


def pm_power_spectrum(ctx, nbins):
    k = np.zeros(nbins); pk = np.zeros(nbins); nm = np.zeros(nbins, dtype=np.int64)
    _check(ctx, lib.pm_power_spectrum(ctx, nbins, k.ctypes.data_as(C.POINTER(C.c_double)),
                                      pk.ctypes.data_as(C.POINTER(C.c_double)),
                                      nm.ctypes.data_as(C.POINTER(C.c_int64))))
    return k, pk, nm


def pm_power_spectrum_noalloc(d_pos, n_mesh, omega_m, nbins, stream=None):
    """P(k) of device positions without any device allocation (see include/pm.h for who needs it).

    d_pos must be an (n, 3) float64 CUDA tensor on the current device (or an (n, 3) float64 numpy array, which
    the library rejects as host memory).  Anything else raises ValueError before the library is called: the
    kernels read 3 * n doubles from the pointer, so a flat or FP32 array would be read past its end.
    """
    shape = tuple(getattr(d_pos, "shape", ()))
    if len(shape) != 2 or shape[1] != 3 or shape[0] < 1:
        raise ValueError(f"pm_power_spectrum_noalloc: positions must have shape (n, 3), got {shape}")
    if isinstance(d_pos, np.ndarray):
        if d_pos.dtype != np.float64 or not d_pos.flags["C_CONTIGUOUS"]:
            raise ValueError("pm_power_spectrum_noalloc: positions must be C-contiguous float64")
    else:
        import torch
        if not isinstance(d_pos, torch.Tensor) or d_pos.dtype != torch.float64 or not d_pos.is_contiguous():
            raise ValueError("pm_power_spectrum_noalloc: positions must be a contiguous float64 tensor")
        if not d_pos.is_cuda or d_pos.device.index != torch.cuda.current_device():
            raise ValueError("pm_power_spectrum_noalloc: positions must live on the current CUDA device")
    k = np.zeros(nbins); pk = np.zeros(nbins); nm = np.zeros(nbins, dtype=np.int64)
    n_part = shape[0]
    st = lib.pm_power_spectrum_noalloc(_ptr(d_pos), int(n_part), int(n_mesh), float(omega_m), int(nbins),
                                       k.ctypes.data_as(C.POINTER(C.c_double)),
                                       pk.ctypes.data_as(C.POINTER(C.c_double)),
                                       nm.ctypes.data_as(C.POINTER(C.c_int64)),
                                       getattr(stream, "cuda_stream", stream))
    if st != PM_OK:
        raise PMError(st, "pm_power_spectrum_noalloc failed")
    return k, pk, nm


def pm_get_time(ctx):
    s = C.c_int32(); a = C.c_double(); t = C.c_double()
    _check(ctx, lib.pm_get_time(ctx, C.byref(s), C.byref(a), C.byref(t)))
    return s.value, a.value, t.value


def pm_get_schedule(ctx, n_steps):
    a = np.zeros(n_steps + 1); dt = np.zeros(n_steps); ah = np.zeros(n_steps)
    dp = C.POINTER(C.c_double)
    _check(ctx, lib.pm_get_schedule(ctx, a.ctypes.data_as(dp), dt.ctypes.data_as(dp), ah.ctypes.data_as(dp)))
    return a, dt, ah


def pm_fft_shapes(ctx, force_y=-1, force_z=-1):
    """Select (0..2), keep (-2) or, with -1, time and keep the fastest y / z column-pass shape; returns the
    shapes in use."""
    y, z = C.c_int32(), C.c_int32()
    _check(ctx, lib.pm_fft_shapes(ctx, force_y, force_z, C.byref(y), C.byref(z)))
    return y.value, z.value


# pm_packed_particle: int32 cell, 3 f32 offsets in [0, 1), 3 f32 momenta (28 bytes)
PACKED = np.dtype([("cell", "<i4"), ("f", "<f4", (3,)), ("u", "<f4", (3,))])
assert PACKED.itemsize == 28


def _packed_ptr(a, n):
    """Pointer to n packed records: a numpy array of dtype PACKED or a torch uint8 tensor of 28 n bytes."""
    if isinstance(a, np.ndarray):
        if a.dtype != PACKED or a.size != n or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"packed particles must be a contiguous array of {n} records of dtype PACKED")
        return a.ctypes.data
    if getattr(a, "numel", None) is None or a.numel() * a.element_size() != 28 * n or not a.is_contiguous():
        raise ValueError(f"packed particles must be a contiguous tensor of {28 * n} bytes")
    return a.data_ptr()


def pm_set_particles_packed(ctx, n_part, records):
    _check(ctx, lib.pm_set_particles_packed(ctx, _packed_ptr(records, n_part)))


def pm_put_particles_packed(ctx, n_part, records):
    _check(ctx, lib.pm_put_particles_packed(ctx, _packed_ptr(records, n_part)))


def pm_get_particles_packed(ctx, n_part, records):
    _check(ctx, lib.pm_get_particles_packed(ctx, _packed_ptr(records, n_part)))


def pm_put_particles_packed_async(ctx, n_part, records):
    """Overlapped put: returns at once; `records` (pinned) must stay unchanged until pm_io_wait."""
    _check(ctx, lib.pm_put_particles_packed_async(ctx, _packed_ptr(records, n_part)))


def pm_get_particles_packed_async(ctx, n_part, records):
    """Overlapped get: returns at once; `records` (pinned) holds the state once pm_io_wait returns."""
    _check(ctx, lib.pm_get_particles_packed_async(ctx, _packed_ptr(records, n_part)))


def pm_io_wait(ctx):
    _check(ctx, lib.pm_io_wait(ctx))


def pm_deposit_shape(ctx, force=-1):
    """Select (0, 1), keep (-2) or, with -1, time and keep the faster projection bin shape; returns the shape
    in use."""
    v = C.c_int32()
    _check(ctx, lib.pm_deposit_shape(ctx, int(force), C.byref(v)))
    return v.value


def pm_get_timings(ctx):
    """Mean per-kernel ms over the steps since the previous call, and the kernel launch count."""
    ms = np.zeros(len(TIMINGS))
    nl = C.c_int64()
    _check(ctx, lib.pm_get_timings(ctx, ms.ctypes.data_as(C.POINTER(C.c_double)), len(TIMINGS), C.byref(nl)))
    return dict(zip(TIMINGS, ms.tolist())), nl.value


def pm_save(ctx, path):
    _check(ctx, lib.pm_save(ctx, os.fsencode(path)))


def pm_load(ctx, path):
    _check(ctx, lib.pm_load(ctx, os.fsencode(path)))


def _echeck(e, st):
    if st != PM_OK:
        raise PMError(st, lib.pm_ensemble_last_error(e).decode() if e else "")


def pm_ensemble_init(configs):
    """configs: list of dicts with the PM() keyword arguments (n_mesh, n_part, box_mpch, omega_m, z_init,
    z_final, n_steps, precision, flags)."""
    arr = (pm_config * len(configs))()
    for i, c in enumerate(configs):
        arr[i] = pm_config(int(c["n_mesh"]), int(c.get("n_steps", 100)), int(c["n_part"]), float(c["box_mpch"]),
                           float(c["omega_m"]), float(c["z_init"]), float(c.get("z_final", 0.0)),
                           int(c.get("precision", PM_FP64)), int(c.get("flags", 0)), None)
    h = C.c_void_p()
    st = lib.pm_ensemble_init(C.cast(arr, C.c_void_p), len(configs), C.byref(h))
    if st != PM_OK:
        raise PMError(st, "pm_ensemble_init failed")
    return h.value


def pm_ensemble_destroy(e):
    lib.pm_ensemble_destroy(e)


def pm_ensemble_last_error(e):
    return lib.pm_ensemble_last_error(e).decode()


def pm_ensemble_box(e, box):
    h = C.c_void_p()
    _echeck(e, lib.pm_ensemble_box(e, int(box), C.byref(h)))
    return h.value


def pm_ensemble_set_particles(e, box, pos, mom):
    _echeck(e, lib.pm_ensemble_set_particles(e, int(box), _ptr(pos), _ptr(mom)))


def pm_ensemble_step(e, use_graph=True):
    _echeck(e, lib.pm_ensemble_step(e, int(bool(use_graph))))


def pm_ensemble_sync(e):
    _echeck(e, lib.pm_ensemble_sync(e))


def pm_ensemble_stream(e):
    """The ensemble's stream handle (an int usable as torch.cuda.ExternalStream(handle))."""
    h = C.c_void_p()
    _echeck(e, lib.pm_ensemble_stream(e, C.byref(h)))
    return h.value or 0


def pm_ensemble_set_streams(e, n_streams):
    _echeck(e, lib.pm_ensemble_set_streams(e, int(n_streams)))


def pm_ensemble_set_batched(e, batched):
    _echeck(e, lib.pm_ensemble_set_batched(e, int(bool(batched))))


def pm_ensemble_get_mode(e):
    """(stream count, batched flag) in use."""
    k, b = C.c_int32(), C.c_int32()
    _echeck(e, lib.pm_ensemble_get_mode(e, C.byref(k), C.byref(b)))
    return k.value, bool(b.value)


def pm_ensemble_tune(e):
    k = C.c_int32()
    _echeck(e, lib.pm_ensemble_tune(e, C.byref(k)))
    return k.value


# ---- learned force correction ---------------------------------------------------------------------

PM_NET_INPUT, PM_NET_OUTPUT, PM_NET_GRAD = 0, 1, 2


def _ncheck(net, st):
    if st != PM_OK:
        raise PMError(st, lib.pm_net_last_error(net).decode() if net else "")


def pm_net_param_count():
    return int(lib.pm_net_param_count())


def pm_net_create(n_mesh, seed=0, stream=None):
    h = C.c_void_p()
    st = lib.pm_net_create(int(n_mesh), C.c_uint64(int(seed)), _stream(stream), C.byref(h))
    if st != PM_OK:
        raise PMError(st, "pm_net_create failed")
    return h.value


def pm_net_destroy(net):
    lib.pm_net_destroy(net)


def pm_net_last_error(net):
    return lib.pm_net_last_error(net).decode()


def pm_net_set_params(net, params):
    _ncheck(net, lib.pm_net_set_params(net, _ptr(params)))


def pm_net_get_params(net, params):
    _ncheck(net, lib.pm_net_get_params(net, _ptr(params)))


def pm_net_buffer(net, which):
    h = C.c_void_p()
    _ncheck(net, lib.pm_net_buffer(net, int(which), C.byref(h)))
    return h.value


def pm_net_features(net, ctx):
    _ncheck(net, lib.pm_net_features(net, ctx))


def pm_net_target(net, coarse, fine, target):
    _ncheck(net, lib.pm_net_target(net, coarse, fine, _ptr(target)))


def pm_net_forward(net):
    _ncheck(net, lib.pm_net_forward(net))


def pm_net_backward(net, target, want_loss=True):
    loss = C.c_double(0.0)
    _ncheck(net, lib.pm_net_backward(net, _ptr(target), C.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def pm_net_adam(net, lr):
    _ncheck(net, lib.pm_net_adam(net, C.c_float(lr)))


def pm_net_train_step(net, target, lr, want_loss=True):
    loss = C.c_double(0.0)
    _ncheck(net, lib.pm_net_train_step(net, _ptr(target), C.c_float(lr), C.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def pm_net_apply(net, ctx):
    _ncheck(net, lib.pm_net_apply(net, ctx))


def pm_net_set_scales(net, s_delta, s_phi, s_target):
    _ncheck(net, lib.pm_net_set_scales(net, float(s_delta), float(s_phi), float(s_target)))


def pm_set_correction(ctx, corr):
    _check(ctx, lib.pm_set_correction(ctx, _ptr(corr)))


def pm_conv3d_forward(n, x, w, bias, c_out, relu, y, stream=None):
    st = lib.pm_conv3d_forward(int(n), _ptr(x), _ptr(w), _ptr(bias), int(c_out), int(relu), _ptr(y), _stream(stream))
    if st != PM_OK:
        raise PMError(st, "pm_conv3d_forward failed")


def pm_conv3d_backward_weight(n, x, g, dw, stream=None):
    st = lib.pm_conv3d_backward_weight(int(n), _ptr(x), _ptr(g), _ptr(dw), _stream(stream))
    if st != PM_OK:
        raise PMError(st, "pm_conv3d_backward_weight failed")


def pm_conv3d_check(stream=None):
    """Raise PMError(PM_ERR_TIMEOUT) if a bounded wait of the tensor-core convolution ran out since the last check."""
    st = lib.pm_conv3d_check(_stream(stream))
    if st != PM_OK:
        raise PMError(st, "pm_conv3d_check: " + STATUS_NAMES.get(st, str(st)))


class PM:
    """Convenience owner of one context; all methods call the functions above."""

    def __init__(self, n_mesh, n_part, box_mpch, omega_m, z_init, z_final=0.0, n_steps=100, precision=PM_FP64,
                 flags=0, stream=None):
        self.n = int(n_mesh)
        self.np = int(n_part)
        self.n_steps = int(n_steps)
        self.ctx = pm_init(n_mesh, n_part, box_mpch, omega_m, z_init, z_final, n_steps, precision, flags, stream)

    def close(self):
        if self.ctx:
            pm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, pos, mom):
        pm_set_particles(self.ctx, pos, mom)

    def put_particles(self, pos, mom):
        pm_put_particles(self.ctx, pos, mom)

    def step(self):
        pm_step(self.ctx)

    def step_graph(self, on=True):
        pm_step_graph(self.ctx, 1 if on else 0)

    def project(self):
        pm_project(self.ctx)

    def solve(self):
        pm_solve(self.ctx)

    def update(self):
        pm_update(self.ctx)

    def particles(self):
        pos = np.zeros((self.np, 3)); mom = np.zeros((self.np, 3))
        pm_get_particles(self.ctx, pos, mom)
        return pos, mom

    def field(self, name):
        out = np.zeros((self.n, self.n, self.n))
        pm_get_field(self.ctx, name, out)
        return out

    def tensor(self, name):
        out = np.zeros(2 * self.n * self.n * (self.n // 2 + 1))
        pm_get_tensor(self.ctx, name, out)
        return out.view(np.complex128).reshape(self.n, self.n, self.n // 2 + 1)

    def power_spectrum(self, nbins):
        return pm_power_spectrum(self.ctx, nbins)

    def time(self):
        return pm_get_time(self.ctx)

    def schedule(self):
        return pm_get_schedule(self.ctx, self.n_steps)

    def timings(self):
        return pm_get_timings(self.ctx)

    def save(self, path):
        pm_save(self.ctx, path)

    def load(self, path):
        pm_load(self.ctx, path)
