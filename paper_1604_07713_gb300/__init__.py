"""gbpic: GB300-native electrostatic PIC-MCC on a cell-based adaptive quadtree.

Thin ctypes binding of the C ABI in ``include/gbpic.h`` (same function names, argument
marshalling only).  Every step of the particle cycle runs in the CUDA kernels of
``lib/libgbpic.so``; there is no CPU fallback: importing works without the library, but any
call raises ``RuntimeError`` when it has not been built (``build()``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgbpic.so")

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ESTATE, PIC_ECAPACITY, PIC_ETIMEOUT, \
    PIC_ENOTCONV, PIC_WARN_STABILITY = range(9)
STATUS_NAMES = ["PIC_OK", "PIC_EINVAL", "PIC_ENOMEM", "PIC_ECUDA", "PIC_ESTATE", "PIC_ECAPACITY",
                "PIC_ETIMEOUT", "PIC_ENOTCONV", "PIC_WARN_STABILITY"]
PIC_FP32, PIC_FP64 = 0, 1
PIC_BC_PERIODIC, PIC_BC_DIRICHLET, PIC_BC_NEUMANN = 0, 1, 2
PIC_ADAPT_MESH, PIC_ADAPT_PARTICLES = 1, 2
PIC_FIELD_PHI, PIC_FIELD_RHO, PIC_FIELD_COUNT_E, PIC_FIELD_COUNT_I, PIC_FIELD_NODE_E, \
    PIC_FIELD_EMAG, PIC_FIELD_AVG_NE, PIC_FIELD_AVG_NI, PIC_FIELD_AVG_TE, PIC_FIELD_AVG_PHI = range(10)
PHASES = ["deposit", "poisson", "node_e", "lists", "scan", "move", "sort", "adapt", "split_merge", "graph"]
PIC_N_PHASES = len(PHASES)

EXPORTED = ["pic_create", "pic_destroy", "pic_set_stream", "pic_set_mesh", "pic_load_particles",
            "pic_step", "pic_compute_fields", "pic_adapt", "pic_read_fields", "pic_read_mesh",
            "pic_read_particles", "pic_get_counts", "pic_get_step", "pic_set_step",
            "pic_set_timing", "pic_get_timing", "pic_get_launch_count", "pic_get_list_stats", "pic_read_emag_noalloc",
            "pic_autotune", "pic_get_tuning", "pic_stability_limits", "pic_check_stability",
            "pic_checkpoint_write", "pic_checkpoint_read", "pic_inject_fault", "pic_diag_enable",
            "pic_diag_reset", "pic_read_eedf", "pic_last_error"]
PIC_FAULT_NONE, PIC_FAULT_ALLOC, PIC_FAULT_BALANCE = 0, 1, 2
PIC_SHAPE_NGP, PIC_SHAPE_CIC_EM, PIC_SHAPE_CIC_EC = 0, 1, 2


class PicConfig(C.Structure):
    """Mirror of ``pic_config`` (include/gbpic.h)."""
    _fields_ = [
        ("precision", C.c_int32), ("n_species", C.c_int32), ("seed", C.c_uint64),
        ("dt", C.c_double), ("eps0", C.c_double), ("q", C.c_double * 2), ("m", C.c_double * 2),
        ("qe", C.c_double), ("mcc", C.c_int32), ("bc_x", C.c_int32), ("bc_y", C.c_int32),
        ("max_level", C.c_int32), ("gas_density", C.c_double), ("gas_temperature_ev", C.c_double),
        ("neutral_mass", C.c_double), ("sigma_el", C.c_double), ("sigma_iz0", C.c_double),
        ("eps_th_ev", C.c_double), ("phi_left_dc", C.c_double), ("phi_left_amp", C.c_double),
        ("phi_left_freq", C.c_double), ("phi_right", C.c_double), ("rho_background", C.c_double),
        ("ppc_target", C.c_int32), ("ppc_min", C.c_int32), ("ppc_max", C.c_int32),
        ("adapt_every", C.c_int32), ("e_ref", C.c_double), ("refine_field", C.c_double),
        ("coarsen_field", C.c_double), ("refine_count", C.c_int32), ("coarsen_count", C.c_int32),
        ("mg_rel_tol", C.c_double), ("mg_max_cycles", C.c_int32), ("instance", C.c_int32),
        ("particle_capacity", C.c_int64), ("shape", C.c_int32), ("implicit", C.c_int32),
    ]


def config_struct(cfg: dict) -> PicConfig:
    c = PicConfig()
    for name, typ in PicConfig._fields_:
        if name not in cfg:
            continue
        v = cfg[name]
        if name in ("q", "m"):
            arr = (C.c_double * 2)(*(list(v) + [0.0] * (2 - len(v))))
            setattr(c, name, arr)
        else:
            setattr(c, name, v)
    return c


_lib = None


class PicError(RuntimeError):
    def __init__(self, fn, status, msg):
        self.status = status
        super().__init__(f"{fn} -> {STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")


def build(force: bool = False) -> str:
    from . import _build as _b
    return _b.build(force=force)


def lib():
    """The loaded CUDA library.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"gbpic CUDA library missing at {LIB_PATH}: run "
                               "paper_1604_07713_gb300.build() (needs nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        _declare(L)
        _lib = L
    return _lib


_p = C.c_void_p
_i32, _i64 = C.c_int32, C.c_int64


def _declare(L):
    sig = {
        "pic_create": [_p, _i32, _p], "pic_destroy": [_p], "pic_set_stream": [_p, _p],
        "pic_set_mesh": [_p, _i32, _i32, _i32, C.c_double, _i64, _p, _p, _p],
        "pic_load_particles": [_p, _i32, _i32, _i64, _p, _p, _p, _p, _p, _p, _p],
        "pic_step": [_p, _i32], "pic_compute_fields": [_p], "pic_adapt": [_p, _i32],
        "pic_read_fields": [_p, _i32, _i32, _p, _i64, _p],
        "pic_read_mesh": [_p, _i32, _p, _p, _p, _i64, _p],
        "pic_read_particles": [_p, _i32, _i32, _p, _p, _p, _p, _p, _p, _p, _p, _i64, _p],
        "pic_get_counts": [_p, _i32, _p, _p, _p, _p, _p], "pic_get_step": [_p, _p],
        "pic_set_step": [_p, _i64], "pic_set_timing": [_p, _i32],
        "pic_get_timing": [_p, _p, _p, _i32], "pic_get_launch_count": [_p, _p],
        "pic_get_list_stats": [_p, _i32, _i32, _p, _p, _p],
        "pic_read_emag_noalloc": [_p, _i32, _p, _i64, _p],
        "pic_autotune": [_p, _i32, _p], "pic_get_tuning": [_p, _p, _p, _p, _p, _p],
        "pic_stability_limits": [_p, C.c_double, C.c_double, C.c_double, _p, _p],
        "pic_check_stability": [_p, _i32, _p, _p, _p],
        "pic_checkpoint_write": [_p, _i32, _p, _i64, _p], "pic_checkpoint_read": [_p, _i32, _p, _i64],
        "pic_inject_fault": [_p, _i32, _i64],
        "pic_diag_enable": [_p, _i32, _i32, C.c_double, _p], "pic_diag_reset": [_p, _i32],
        "pic_read_eedf": [_p, _i32, _p, _i64, _p, _p],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.pic_last_error.argtypes = []
    L.pic_last_error.restype = C.c_char_p


def _call(name, *args, ok=(PIC_OK,)):
    st = getattr(lib(), name)(*args)
    if st not in ok:
        raise PicError(name, st, lib().pic_last_error().decode())
    return st


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------------------
# Functions with the C ABI's names
# ---------------------------------------------------------------------------------------
def pic_create(cfgs) -> C.c_void_p:
    if isinstance(cfgs, dict):
        cfgs = [cfgs]
    arr = (PicConfig * len(cfgs))(*[config_struct(c) for c in cfgs])
    out = C.c_void_p()
    _call("pic_create", C.cast(arr, C.c_void_p), len(cfgs), C.byref(out))
    return out


def pic_destroy(ctx):
    lib().pic_destroy(ctx)


def pic_set_stream(ctx, stream_handle: int):
    _call("pic_set_stream", ctx, C.c_void_p(stream_handle))


def pic_set_mesh(ctx, inst, nx0, ny0, h0, root=None, morton=None, level=None):
    if root is None:
        n = nx0 * ny0
        _call("pic_set_mesh", ctx, inst, nx0, ny0, h0, n, None, None, None)
        return
    r = np.ascontiguousarray(root, np.uint32)
    m = np.ascontiguousarray(morton, np.uint32)
    lv = np.ascontiguousarray(level, np.uint8)
    _call("pic_set_mesh", ctx, inst, nx0, ny0, h0, r.size, _ptr(r), _ptr(m), _ptr(lv))


def pic_load_particles(ctx, inst, species, x, y, vx, vy, vz, w, ids=None):
    """Returns PIC_OK, or PIC_WARN_STABILITY when the loaded electrons break the explicit-PIC
    limits (the particles are loaded either way)."""
    arrs = [_f64(a) for a in (x, y, vx, vy, vz, w)]
    n = arrs[0].size
    i = None if ids is None else np.ascontiguousarray(ids, np.uint64)
    return _call("pic_load_particles", ctx, inst, species, n, *[_ptr(a) for a in arrs], _ptr(i),
                 ok=(PIC_OK, PIC_WARN_STABILITY))


def pic_step(ctx, n_steps=1, allow_notconv=False):
    return _call("pic_step", ctx, n_steps, ok=(PIC_OK, PIC_ENOTCONV) if allow_notconv else (PIC_OK,))


def pic_compute_fields(ctx, allow_notconv=False):
    return _call("pic_compute_fields", ctx, ok=(PIC_OK, PIC_ENOTCONV) if allow_notconv else (PIC_OK,))


def pic_adapt(ctx, flags=PIC_ADAPT_MESH | PIC_ADAPT_PARTICLES):
    _call("pic_adapt", ctx, flags)


def pic_read_fields(ctx, inst, field):
    n = C.c_int64()
    st = lib().pic_read_fields(ctx, inst, field, None, 0, C.byref(n))
    if st not in (PIC_OK, PIC_EINVAL) or n.value <= 0:
        raise PicError("pic_read_fields", st, lib().pic_last_error().decode())
    out = np.empty(n.value, np.float64)
    _call("pic_read_fields", ctx, inst, field, _ptr(out), out.size, C.byref(n))
    return out.reshape(-1, 4, 2) if field == PIC_FIELD_NODE_E else out


def pic_read_mesh(ctx, inst):
    n = C.c_int64()
    lib().pic_read_mesh(ctx, inst, None, None, None, 0, C.byref(n))
    r = np.empty(n.value, np.uint32); m = np.empty(n.value, np.uint32); lv = np.empty(n.value, np.uint8)
    _call("pic_read_mesh", ctx, inst, _ptr(r), _ptr(m), _ptr(lv), n.value, C.byref(n))
    return r, m, lv


def pic_read_particles(ctx, inst, species):
    n = C.c_int64()
    lib().pic_read_particles(ctx, inst, species, *([None] * 8), 0, C.byref(n))
    k = n.value
    out = {name: np.empty(k, np.float64) for name in ("x", "y", "vx", "vy", "vz", "w")}
    out["id"] = np.empty(k, np.uint64)
    out["leaf"] = np.empty(k, np.uint32)
    _call("pic_read_particles", ctx, inst, species, *[_ptr(out[nm]) for nm in ("x", "y", "vx", "vy", "vz", "w")],
          _ptr(out["id"]), _ptr(out["leaf"]), k, C.byref(n))
    return out


def pic_get_counts(ctx, inst=0):
    nl, ne, ni = C.c_int64(), C.c_int64(), C.c_int64()
    cyc, res = C.c_int32(), C.c_double()
    _call("pic_get_counts", ctx, inst, C.byref(nl), C.byref(ne), C.byref(ni), C.byref(cyc), C.byref(res))
    return dict(n_leaves=nl.value, n_e=ne.value, n_i=ni.value, mg_cycles=cyc.value, mg_rel_res=res.value)


def pic_get_step(ctx):
    s = C.c_int64()
    _call("pic_get_step", ctx, C.byref(s))
    return s.value


def pic_set_step(ctx, step):
    _call("pic_set_step", ctx, step)


def pic_set_timing(ctx, on=True):
    _call("pic_set_timing", ctx, 1 if on else 0)


def pic_get_timing(ctx):
    ms = np.zeros(PIC_N_PHASES); ln = np.zeros(PIC_N_PHASES, np.int64)
    _call("pic_get_timing", ctx, _ptr(ms), _ptr(ln), PIC_N_PHASES)
    return {p: (float(ms[i]), int(ln[i])) for i, p in enumerate(PHASES)}


def pic_get_list_stats(ctx, inst=0, species=0):
    """(relayouts, tail_moves, overflowed records) of one species' cell lists since its load."""
    r, m, o = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    _call("pic_get_list_stats", ctx, inst, species, C.byref(r), C.byref(m), C.byref(o))
    return r.value, m.value, o.value


def pic_autotune(ctx, max_steps, allow_notconv=False):
    """Run up to max_steps steps, one launch configuration each; keep the fastest.  Returns the
    steps run."""
    used = C.c_int32(0)
    _call("pic_autotune", ctx, max_steps, C.byref(used),
          ok=(PIC_OK, PIC_ENOTCONV) if allow_notconv else (PIC_OK,))
    return used.value


def pic_get_tuning(ctx):
    """The launch configuration in use: push block size, push blocks per SM (256-thread units,
    0 = all resident), the GPU share of a push inside a captured ensemble step (1 / div), the
    captured step's parallel branches, and the best step time the tuner measured (ms)."""
    nt, bps, div, br = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    ms = C.c_double()
    _call("pic_get_tuning", ctx, C.byref(nt), C.byref(bps), C.byref(div), C.byref(br), C.byref(ms))
    return dict(push_threads=nt.value, push_blocks_per_sm=bps.value, graph_push_div=div.value,
                graph_branches=br.value, best_step_ms=ms.value)


def pic_get_launch_count(ctx):
    n = C.c_int64()
    _call("pic_get_launch_count", ctx, C.byref(n))
    return n.value


def pic_read_emag_noalloc(ctx, inst, out: np.ndarray) -> int:
    """|E| per leaf into the caller's FP64 array without any device allocation (fixed
    1 MiB scratch: at most 131,072 leaves).  Returns the number of leaves written."""
    n = C.c_int64()
    _call("pic_read_emag_noalloc", ctx, inst, _ptr(out), out.size, C.byref(n))
    return n.value


def pic_stability_limits(cfg: dict, n_e_max, w_leaf_max, t_e_ev):
    """(status, max h / lambda_D, max omega_pe dt) for the given plasma parameters (host only)."""
    c = config_struct(cfg)
    a, b = C.c_double(), C.c_double()
    st = _call("pic_stability_limits", C.byref(c), n_e_max, w_leaf_max, t_e_ev, C.byref(a), C.byref(b),
               ok=(PIC_OK, PIC_WARN_STABILITY))
    return st, a.value, b.value


def pic_check_stability(ctx, inst=0):
    """(status, max h / lambda_D, max omega_pe dt, T_e [eV]) of the instance's electrons."""
    a, b, t = C.c_double(), C.c_double(), C.c_double()
    st = _call("pic_check_stability", ctx, inst, C.byref(a), C.byref(b), C.byref(t),
               ok=(PIC_OK, PIC_WARN_STABILITY))
    return st, a.value, b.value, t.value


def pic_checkpoint_write(ctx, inst=0) -> bytes:
    n = C.c_int64()
    lib().pic_checkpoint_write(ctx, inst, None, 0, C.byref(n))
    if n.value <= 0:
        raise PicError("pic_checkpoint_write", PIC_EINVAL, lib().pic_last_error().decode())
    buf = C.create_string_buffer(n.value)
    _call("pic_checkpoint_write", ctx, inst, C.cast(buf, C.c_void_p), n.value, C.byref(n))
    return buf.raw[:n.value]


def pic_checkpoint_read(ctx, inst, image: bytes):
    buf = C.create_string_buffer(image, len(image))
    _call("pic_checkpoint_read", ctx, inst, C.cast(buf, C.c_void_p), len(image))


def pic_diag_enable(ctx, inst, n_bins, eps_max_ev, region=None):
    r = None if region is None else np.ascontiguousarray(region, np.float64)
    _call("pic_diag_enable", ctx, inst, n_bins, eps_max_ev, _ptr(r))


def pic_diag_reset(ctx, inst=0):
    _call("pic_diag_reset", ctx, inst)


def pic_read_eedf(ctx, inst=0):
    """(f [1/eV] per energy bin, steps accumulated)."""
    n, k = C.c_int64(), C.c_int64()
    lib().pic_read_eedf(ctx, inst, None, 0, C.byref(n), None)
    out = np.empty(max(0, n.value), np.float64)
    _call("pic_read_eedf", ctx, inst, _ptr(out), out.size, C.byref(n), C.byref(k))
    return out, k.value


def pic_inject_fault(ctx, kind, count=0):
    _call("pic_inject_fault", ctx, kind, count)


def pic_last_error() -> str:
    return lib().pic_last_error().decode()


# ---------------------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------------------
class Context:
    """Owns one pic_ctx; methods forward to the functions above."""

    def __init__(self, cfgs, stream_handle: int | None = None):
        self.cfgs = [cfgs] if isinstance(cfgs, dict) else list(cfgs)
        self.ctx = pic_create(self.cfgs)
        if stream_handle is not None:
            pic_set_stream(self.ctx, stream_handle)

    def close(self):
        if self.ctx is not None:
            pic_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mesh(self, inst=0, nx0=1, ny0=1, h0=1.0, root=None, morton=None, level=None, lmax=None):
        pic_set_mesh(self.ctx, inst, nx0, ny0, h0, root, morton, level)

    def set_mesh_dict(self, mesh: dict, inst=0):
        pic_set_mesh(self.ctx, inst, mesh["nx0"], mesh["ny0"], mesh["h0"], mesh.get("root"),
                     mesh.get("morton"), mesh.get("level"))

    def load(self, species, x, y, vx, vy, vz, w, ids=None, inst=0):
        return pic_load_particles(self.ctx, inst, species, x, y, vx, vy, vz, w, ids)

    def checkpoint(self, inst=0) -> bytes:
        return pic_checkpoint_write(self.ctx, inst)

    def restore(self, image: bytes, inst=0):
        pic_checkpoint_read(self.ctx, inst, image)

    def stability(self, inst=0):
        return pic_check_stability(self.ctx, inst)

    def diag_enable(self, n_bins, eps_max_ev, region=None, inst=0):
        pic_diag_enable(self.ctx, inst, n_bins, eps_max_ev, region)

    def eedf(self, inst=0):
        return pic_read_eedf(self.ctx, inst)

    def step(self, n=1, allow_notconv=False):
        return pic_step(self.ctx, n, allow_notconv)

    def compute_fields(self, allow_notconv=False):
        return pic_compute_fields(self.ctx, allow_notconv)

    def adapt(self, flags=PIC_ADAPT_MESH | PIC_ADAPT_PARTICLES):
        pic_adapt(self.ctx, flags)

    def fields(self, field, inst=0):
        return pic_read_fields(self.ctx, inst, field)

    def mesh(self, inst=0):
        return pic_read_mesh(self.ctx, inst)

    def particles(self, species, inst=0):
        return pic_read_particles(self.ctx, inst, species)

    def counts(self, inst=0):
        return pic_get_counts(self.ctx, inst)

    def autotune(self, max_steps=12, allow_notconv=False):
        return pic_autotune(self.ctx, max_steps, allow_notconv)

    def tuning(self):
        return pic_get_tuning(self.ctx)
