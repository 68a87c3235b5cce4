"""ctypes binding of the C ABI in include/icon.h (argument marshalling only).

Every function here has the name of the C entry point it calls; all computation
happens in the CUDA library. Errors raise IconError with the library's message.
If the compiled library is missing the import fails: there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libicon_gb300.so")

ICON_OK, ICON_EINVAL, ICON_ENOMEM, ICON_ECUDA, ICON_ETIMEOUT, ICON_ENONFINITE, ICON_EINDEX = range(7)
STATUS_NAMES = {0: "ICON_OK", 1: "ICON_EINVAL", 2: "ICON_ENOMEM", 3: "ICON_ECUDA", 4: "ICON_ETIMEOUT",
                5: "ICON_ENONFINITE", 6: "ICON_EINDEX"}
ICON_FP64, ICON_MIXED = 0, 1
ICON_CASE_REST, ICON_CASE_SBR, ICON_CASE_JET, ICON_CASE_MEMBER = 0, 1, 2, 3

# table ids: name -> (id, dtype, entity ('c','e','v'), columns)
TABLES = {
    "c2v": (0, np.int32, "c", 3), "c2e": (1, np.int32, "c", 3), "e2c": (2, np.int32, "e", 2),
    "e2v": (3, np.int32, "e", 2), "v2e": (4, np.int32, "v", 6), "v2c": (5, np.int32, "v", 6),
    "vdeg": (6, np.int32, "v", 1), "e2vt": (7, np.int32, "e", 5), "e2q": (8, np.int32, "e", 4),
    "x_c": (16, np.float64, "c", 3), "x_e": (17, np.float64, "e", 3), "x_v": (18, np.float64, "v", 3),
    "n_e": (19, np.float64, "e", 3), "t_e": (20, np.float64, "e", 3), "l_e": (21, np.float64, "e", 1),
    "d_e": (22, np.float64, "e", 1), "A_c": (23, np.float64, "c", 1), "A_v": (24, np.float64, "v", 1),
    "f_e": (25, np.float64, "e", 1), "vt_w": (26, np.float64, "e", 5), "kin_w": (27, np.float64, "c", 3),
    "lsq_w": (28, np.float64, "v", 18), "L34": (29, np.float64, "e", 1), "s_ce": (30, np.float64, "c", 3),
    "s_ve": (31, np.float64, "v", 6),
    # tracer transport tables (built on demand)
    "c2c": (9, np.int32, "c", 3), "lsq_c": (32, np.float64, "c", 9), "roff": (33, np.float64, "e", 6),
}
# field ids: name -> (id, entity, half-level field)
FIELDS = {"vn": (0, "e", False), "w": (1, "c", True), "rho": (2, "c", False), "theta_v": (3, "c", False),
          "exner": (4, "c", False), "mflx": (5, "e", False), "wflx": (6, "c", True)}


class IconError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class CaseParams(ctypes.Structure):
    _fields_ = [("noise_K", ctypes.c_double), ("top_m", ctypes.c_double), ("stretch_s", ctypes.c_double),
                ("damp_m", ctypes.c_double), ("precision", ctypes.c_int), ("member", ctypes.c_int),
                ("topo_height_m", ctypes.c_double), ("topo_radius_m", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("the CUDA library %s is not built; run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    I64p = ctypes.POINTER(ctypes.c_int64)
    sig = {
        "icon_set_allocator": (I, [P, P, P]), "icon_set_stream": (I, [P]),
        "icon_last_error": (ctypes.c_char_p, []),
        "icon_grid_build": (I, [I, I, I, ctypes.POINTER(P)]),
        "icon_grid_counts": (I, [P, I64p, I64p, I64p]),
        "icon_grid_copy_table": (I, [P, I, P, S]), "icon_grid_free": (None, [P]),
        "icon_state_init": (I, [P, ctypes.c_uint64, I, ctypes.POINTER(P)]),
        "icon_state_init_ex": (I, [P, ctypes.c_uint64, I, ctypes.POINTER(CaseParams), ctypes.POINTER(P)]),
        "icon_dycore_step": (I, [P, D, I]), "icon_dycore_step_async": (I, [P, D, I]),
        "icon_state_status": (I, [P]),
        "icon_global_mass": (I, [P, ctypes.POINTER(D)]), "icon_global_mass_async": (I, [P, P]),
        "icon_state_step_kernels": (I, [P, D, I, ctypes.POINTER(I)]),
        "icon_dycore_step_profile": (I, [P, D, I, ctypes.POINTER(D), ctypes.POINTER(I)]),
        "icon_kernel_kind_name": (ctypes.c_char_p, [I]),
        "icon_selftest": (I, [ctypes.c_longlong, ctypes.POINTER(ctypes.c_uint)]),
        "icon_probe_fp64_rate": (I, [ctypes.POINTER(D), ctypes.POINTER(D)]),
        "icon_partition_plan": (I, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, I, I, I,
                                    I64p, P, P, P]),
        "icon_domain_create": (I, [P, I, I, ctypes.POINTER(P)]),
        "icon_domain_step": (I, [P, D, I]),
        "icon_domain_global_mass": (I, [P, ctypes.POINTER(D)]),
        "icon_domain_copy_field": (I, [P, I, P, S]),
        "icon_domain_part_counts": (I, [P, I, I64p]),
        "icon_domain_free": (None, [P]),
        "icon_global_mass_noalloc": (I, [P, P, P, I, ctypes.POINTER(D)]),
        "icon_state_copy_field": (I, [P, I, P, S]), "icon_state_set_field": (I, [P, I, P, S]),
        "icon_state_precision": (I, [P, ctypes.POINTER(I)]), "icon_state_free": (None, [P]),
        "icon_ensemble_create": (I, [ctypes.POINTER(P), I, ctypes.POINTER(P)]),
        "icon_ensemble_step": (I, [P, ctypes.POINTER(D), I, I]), "icon_ensemble_free": (None, [P]),
        "icon_ensemble_set_option": (I, [P, I, ctypes.c_longlong]),
        "icon_ensemble_step_profile": (I, [P, ctypes.POINTER(D), I, ctypes.POINTER(D), ctypes.POINTER(I)]),
        "icon_ensemble_phase_name": (ctypes.c_char_p, [I]),
        "icon_state_tiling": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "icon_state_set_tiling": (I, [P, I, I, I]),
        "icon_state_set_option": (I, [P, I, D]),
        "icon_state_add_tracers": (I, [P, I]), "icon_state_tracers": (I, [P, ctypes.POINTER(I)]),
        "icon_state_set_tracer": (I, [P, I, P, S]), "icon_state_copy_tracer": (I, [P, I, P, S]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
DEALLOC_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_keep = []


def _check(rc):
    if rc != ICON_OK:
        raise IconError(rc, _lib.icon_last_error().decode())


def exported_symbols():
    """Names of the C entry points this binding resolved (all of include/icon.h)."""
    return sorted(n for n in dir(_lib) if n.startswith("icon_"))


# ---------------------------------------------------------------- allocator / stream
def icon_set_allocator(alloc, dealloc):
    """Register Python callables alloc(nbytes) -> int device pointer and dealloc(ptr);
    (None, None) restores cudaMalloc."""
    if alloc is None:
        _check(_lib.icon_set_allocator(None, None, None))
        return
    def _alloc(n, ctx):
        # an exception escaping a ctypes callback leaves its return value undefined:
        # every failure must come back as NULL
        try:
            return alloc(n) or None
        except Exception:
            return None

    def _dealloc(p, ctx):
        try:
            dealloc(p)
        except Exception:
            pass

    a = ALLOC_FN(_alloc)
    d = DEALLOC_FN(_dealloc)
    _keep.append((a, d))
    _check(_lib.icon_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(d, ctypes.c_void_p), None))


def icon_set_stream(stream_handle):
    _check(_lib.icon_set_stream(ctypes.c_void_p(stream_handle or None)))


# ---------------------------------------------------------------- grid
def icon_grid_build(root, bisections, nlev):
    h = ctypes.c_void_p()
    _check(_lib.icon_grid_build(root, bisections, nlev, ctypes.byref(h)))
    return h


def icon_grid_counts(grid):
    nc, ne, nv = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.icon_grid_counts(grid, ctypes.byref(nc), ctypes.byref(ne), ctypes.byref(nv)))
    return nc.value, ne.value, nv.value


def icon_grid_copy_table(grid, name):
    tid, dt, ent, cols = TABLES[name]
    nc, ne, nv = icon_grid_counts(grid)
    n = {"c": nc, "e": ne, "v": nv}[ent]
    out = np.empty((n, cols) if cols > 1 else (n,), dtype=dt)
    _check(_lib.icon_grid_copy_table(grid, tid, out.ctypes.data, out.nbytes))
    return out


def icon_grid_free(grid):
    _lib.icon_grid_free(grid)


# ---------------------------------------------------------------- state
def icon_state_init(grid, seed, case_id):
    h = ctypes.c_void_p()
    _check(_lib.icon_state_init(grid, seed, case_id, ctypes.byref(h)))
    return h


def icon_state_init_ex(grid, seed, case_id, noise_K=-1.0, precision=ICON_FP64, member=0,
                       topo_height_m=0.0, topo_radius_m=0.0):
    p = CaseParams(noise_K, -1.0, -1.0, -1.0, precision, member, topo_height_m, topo_radius_m)
    h = ctypes.c_void_p()
    _check(_lib.icon_state_init_ex(grid, seed, case_id, ctypes.byref(p), ctypes.byref(h)))
    return h


def icon_dycore_step(state, dt, nsubsteps):
    _check(_lib.icon_dycore_step(state, dt, nsubsteps))


def icon_dycore_step_async(state, dt, nsubsteps):
    _check(_lib.icon_dycore_step_async(state, dt, nsubsteps))


def icon_state_status(state):
    _check(_lib.icon_state_status(state))


def icon_global_mass(state):
    m = ctypes.c_double()
    _check(_lib.icon_global_mass(state, ctypes.byref(m)))
    return m.value


def icon_global_mass_async(state, host_ptr):
    """Enqueue the mass integral; the result lands in the 8-byte host buffer at host_ptr."""
    _check(_lib.icon_global_mass_async(state, ctypes.c_void_p(host_ptr)))


def icon_global_mass_noalloc(grid, dev_rho_ptr, ld, dev_dz_ptr=0):
    """Mass of a caller-owned device density array [Nc][ld] without any device allocation;
    dev_dz_ptr (optional) the device array of per-cell layer thicknesses in the same layout."""
    m = ctypes.c_double()
    _check(_lib.icon_global_mass_noalloc(grid, ctypes.c_void_p(dev_rho_ptr), ctypes.c_void_p(dev_dz_ptr or None),
                                         ld, ctypes.byref(m)))
    return m.value


def icon_state_step_kernels(state, dt, nsubsteps):
    n = ctypes.c_int()
    _check(_lib.icon_state_step_kernels(state, dt, nsubsteps, ctypes.byref(n)))
    return n.value


ICON_KIND_COUNT = 26


def icon_dycore_step_profile(state, dt, nsubsteps, ms=None, launches=None):
    """One eager step with CUDA events around every launch; returns the accumulated
    (ms per kind, launches per kind) arrays."""
    if ms is None:
        ms = np.zeros(ICON_KIND_COUNT)
        launches = np.zeros(ICON_KIND_COUNT, dtype=np.int32)
    _check(_lib.icon_dycore_step_profile(state, dt, nsubsteps, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         launches.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return ms, launches


def icon_selftest(n):
    f = ctypes.c_uint()
    _check(_lib.icon_selftest(n, ctypes.byref(f)))
    return f.value


def icon_probe_fp64_rate():
    """(FP64 FMA, FP64 ADD) instructions per second measured on the current device."""
    f, a = ctypes.c_double(), ctypes.c_double()
    _check(_lib.icon_probe_fp64_rate(ctypes.byref(f), ctypes.byref(a)))
    return f.value, a.value


def icon_kernel_kind_name(kind):
    n = _lib.icon_kernel_kind_name(kind)
    return n.decode() if n else None


def _field_shape(grid, name, nlev):
    fid, ent, half = FIELDS[name]
    nc, ne, nv = icon_grid_counts(grid)
    return fid, ({"c": nc, "e": ne}[ent], nlev + 1 if half else nlev)


def icon_state_copy_field(state, grid, nlev, name, out=None):
    fid, shape = _field_shape(grid, name, nlev)
    if out is None:
        out = np.empty(shape, dtype=np.float64)
    assert out.shape == shape and out.dtype == np.float64 and out.flags.c_contiguous
    _check(_lib.icon_state_copy_field(state, fid, out.ctypes.data, out.size))
    return out


def icon_state_set_field(state, grid, nlev, name, values):
    fid, shape = _field_shape(grid, name, nlev)
    values = np.ascontiguousarray(values, dtype=np.float64)
    assert values.shape == shape
    _check(_lib.icon_state_set_field(state, fid, values.ctypes.data, values.size))


def icon_state_precision(state):
    p = ctypes.c_int()
    _check(_lib.icon_state_precision(state, ctypes.byref(p)))
    return p.value


def icon_state_free(state):
    _lib.icon_state_free(state)


# ---------------------------------------------------------------- ensemble
def icon_ensemble_create(states):
    arr = (ctypes.c_void_p * len(states))(*[s.value for s in states])
    h = ctypes.c_void_p()
    _check(_lib.icon_ensemble_create(arr, len(states), ctypes.byref(h)))
    return h


def icon_ensemble_step(ens, dts, nsubsteps, nsteps):
    arr = (ctypes.c_double * len(dts))(*dts)
    _check(_lib.icon_ensemble_step(ens, arr, nsubsteps, nsteps))


ICON_ENS_SPIN_LIMIT, ICON_ENS_TEST_SKIP_BARRIER = 1, 2
ICON_ENS_PHASE_COUNT = 14


def icon_ensemble_step_profile(ens, dts, nsubsteps, ms=None, counts=None):
    """One ensemble step with the phase timer; returns the accumulated (ms per phase,
    barriers per phase) arrays."""
    if ms is None:
        ms = np.zeros(ICON_ENS_PHASE_COUNT)
        counts = np.zeros(ICON_ENS_PHASE_COUNT, dtype=np.int32)
    arr = (ctypes.c_double * len(dts))(*dts)
    _check(_lib.icon_ensemble_step_profile(ens, arr, nsubsteps, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return ms, counts


def icon_ensemble_phase_name(phase):
    n = _lib.icon_ensemble_phase_name(phase)
    return n.decode() if n else None
# mixed-precision stencil kinds that take a tile
KIND_MX_VERTEX, KIND_MX_EDGE, KIND_MX_CELL_KE, KIND_MX_EDGE_TEND, KIND_MX_COLUMN_PREP, KIND_MX_DIFF_VERTEX = \
    10, 11, 12, 13, 15, 16
# the lean mixed column: its tile is a launch shape (sweep unroll, resident blocks per SM)
KIND_MX_LEAN = 24
LEAN_SHAPES = ((2, 9), (2, 10), (2, 8), (2, 12), (2, 6))


def icon_ensemble_set_option(ens, option, value):
    _check(_lib.icon_ensemble_set_option(ens, option, value))


def icon_state_tiling(state, kind):
    lanes, block = ctypes.c_int(), ctypes.c_int()
    _check(_lib.icon_state_tiling(state, kind, ctypes.byref(lanes), ctypes.byref(block)))
    return lanes.value, block.value


def icon_state_set_tiling(state, kind, lanes, block):
    _check(_lib.icon_state_set_tiling(state, kind, lanes, block))


def icon_ensemble_free(ens):
    _lib.icon_ensemble_free(ens)


# ---------------------------------------------------------------- tracers
def icon_state_add_tracers(state, n):
    _check(_lib.icon_state_add_tracers(state, n))


def icon_state_tracers(state):
    n = ctypes.c_int()
    _check(_lib.icon_state_tracers(state, ctypes.byref(n)))
    return n.value


def _tracer_shape(grid, nlev):
    nc, _, _ = icon_grid_counts(grid)
    return (nc, nlev)


def icon_state_set_tracer(state, grid, nlev, t, values):
    values = np.ascontiguousarray(values, dtype=np.float64)
    assert values.shape == _tracer_shape(grid, nlev)
    _check(_lib.icon_state_set_tracer(state, t, values.ctypes.data, values.size))


def icon_state_copy_tracer(state, grid, nlev, t):
    out = np.empty(_tracer_shape(grid, nlev), dtype=np.float64)
    _check(_lib.icon_state_copy_tracer(state, t, out.ctypes.data, out.size))
    return out


# ---------------------------------------------------------------- options
ICON_OPT_DIVDAMP4, ICON_OPT_DIFF4, ICON_OPT_UPWIND_THETA = 1, 2, 3


def icon_state_set_option(state, option, value):
    _check(_lib.icon_state_set_option(state, option, float(value)))


# ---------------------------------------------------------------- domain decomposition
def icon_partition_plan(c2e, e2c, c2v, v2c, vdeg, nparts, part, halo_rings):
    """Host-only plan of one part: (counts[6], local ids, owner part, owner index), the
    tables as int32 arrays in the layout of icon_grid_copy_table."""
    arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in (c2e, e2c, c2v, v2c, vdeg)]
    nc, ne, nv = arrs[0].shape[0], arrs[1].shape[0], arrs[4].shape[0]
    counts = np.zeros(6, dtype=np.int64)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    I64p = ctypes.POINTER(ctypes.c_int64)
    _check(_lib.icon_partition_plan(nc, ne, nv, *[ptr(a) for a in arrs], nparts, part, halo_rings,
                                    counts.ctypes.data_as(I64p), None, None, None))
    n = int(counts[3:].sum())
    loc, own, oix = (np.zeros(n, dtype=np.int32) for _ in range(3))
    _check(_lib.icon_partition_plan(nc, ne, nv, *[ptr(a) for a in arrs], nparts, part, halo_rings,
                                    counts.ctypes.data_as(I64p), ptr(loc), ptr(own), ptr(oix)))
    return counts, loc, own, oix


def icon_domain_create(state, nparts, halo_rings):
    h = ctypes.c_void_p()
    _check(_lib.icon_domain_create(state, nparts, halo_rings, ctypes.byref(h)))
    return h


def icon_domain_step(domain, dt, nsubsteps):
    _check(_lib.icon_domain_step(domain, dt, nsubsteps))


def icon_domain_global_mass(domain):
    m = ctypes.c_double()
    _check(_lib.icon_domain_global_mass(domain, ctypes.byref(m)))
    return m.value


def icon_domain_copy_field(domain, grid, nlev, name):
    fid, shape = _field_shape(grid, name, nlev)
    out = np.empty(shape, dtype=np.float64)
    _check(_lib.icon_domain_copy_field(domain, fid, out.ctypes.data, out.size))
    return out


def icon_domain_part_counts(domain, part):
    c = np.zeros(6, dtype=np.int64)
    _check(_lib.icon_domain_part_counts(domain, part, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return c


def icon_domain_free(domain):
    _lib.icon_domain_free(domain)
