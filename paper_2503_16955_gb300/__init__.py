"""GB300-native mosaic-crystal X-ray ray tracer (the per-ray transport of HEART,
arXiv 2503.16955) -- thin Python binding of the C-ABI library libheart.so.

The binding only marshals arguments: every step of the ray path runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  If the
library is missing the calls raise; there is no CPU fallback.

Functions carry the C names of include/heart.h:
    heart_spectrometer_create(desc) -> Spectrometer
    heart_trace(spec, source, n_rays, seed, ray_offset, d_image, precision, stream) -> tally
    heart_trace_host(spec, source, n_rays, seed, ray_offset, h_image, precision) -> tally
    heart_trace_records(spec, source, n_rays, seed, ray_offset, precision, d_image=None) -> (records, tally)
    heart_trace_rays(spec, rays, seed, ray_offset, d_image, precision, records=False) -> tally [, records]
    heart_trace_batch(specs, sources, n_rays, seeds, d_images, stream) -> [tally]
    heart_server_create / heart_submit / heart_poll / heart_release / heart_server_destroy
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libheart.so")

GEOMETRY = {"flat": 0, "cyl": 1}
MDF = {"gaussian": 0, "lorentzian": 1, "pseudo_voigt": 2, "vmf": 3, "wl": 4, "swl": 5, "uniform": 6}
IRC = {"darwin": 0, "darwin_prins": 1, "pseudo_voigt": 2, "gaussian": 3, "lorentzian": 4, "box": 5, "none": 6}
SRC = {"mono": 0, "gauss": 1, "lorentz": 2, "inv_e": 3, "uniform": 4, "table": 5}
PRECISION = {"fp64": 0, "fp32": 1}
COUNT = {"i32": 0, "i64": 1}
SAMPLER = {"thinned": 0, "plain": 1}
STATUS = {0: "HEART_OK", 1: "HEART_EINVAL", 2: "HEART_ENOMEM", 3: "HEART_ECUDA", 4: "HEART_EBUSY",
          5: "HEART_ETIMEOUT", 6: "HEART_ELIMIT", 7: "HEART_ENOTFOUND"}
OUTCOME = {0: "miss", 1: "absorbed", 2: "exit_front", 3: "exit_back", 4: "exit_side",
           5: "capped", 6: "stuck"}

D3 = C.c_double * 3


class heart_spectrometer_desc(C.Structure):
    _fields_ = [
        ("d_spacing_A", C.c_double), ("thickness_mm", C.c_double),
        ("geometry", C.c_int32), ("mdf", C.c_int32), ("radius_mm", C.c_double),
        ("centre_mm", D3), ("normal", D3), ("axis", D3), ("centre_axial_mm", C.c_double),
        ("size_disp_mm", C.c_double), ("size_nondisp_mm", C.c_double),
        ("mdf_fwhm_rad", C.c_double), ("mdf_eta", C.c_double),
        ("irc", C.c_int32), ("max_reflections", C.c_int32),
        ("irc_fwhm_rad", C.c_double), ("irc_lorentz_fwhm_rad", C.c_double),
        ("irc_shift_rad", C.c_double), ("prins_g", C.c_double),
        ("absorption_length_mm", C.c_double), ("absorption_ref_keV", C.c_double),
        ("absorption_power", C.c_double),
        ("refl_K_per_mm2", C.c_double), ("refl_darwin_fwhm_rad", C.c_double), ("refl_ref_keV", C.c_double),
        ("max_collisions", C.c_int64),
        ("det_centre_mm", D3), ("det_u", D3), ("det_v", D3),
        ("det_nx", C.c_int32), ("det_ny", C.c_int32), ("pixel_mm", C.c_double),
        ("count_type", C.c_int32), ("sampler", C.c_int32), ("thin_vstar", C.c_double),
        ("n_orders", C.c_int32), ("reserved2", C.c_int32), ("order_m", C.c_int32 * 4),
        ("order_K_rel", C.c_double * 4), ("order_w_rel", C.c_double * 4),
        ("n_irc_e", C.c_int32), ("reserved3", C.c_int32), ("irc_e_keV", C.c_double * 16),
        ("irc_e_wscale", C.c_double * 16), ("irc_e_shift_rad", C.c_double * 16),
    ]


class heart_spectral_component(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("e0_keV", C.c_double),
                ("width_keV", C.c_double), ("lo_keV", C.c_double), ("hi_keV", C.c_double),
                ("weight", C.c_double)]


class heart_source_desc(C.Structure):
    _fields_ = [("components", C.POINTER(heart_spectral_component)), ("n_components", C.c_int32),
                ("reserved", C.c_int32), ("origin_mm", D3), ("axis", D3),
                ("cone_half_angle_rad", C.c_double), ("spot_fwhm_mm", C.c_double * 2),
                ("polarization", D3), ("table_keV", C.POINTER(C.c_double)),
                ("table_pdf", C.POINTER(C.c_double)), ("n_table", C.c_int32), ("reserved2", C.c_int32)]


class heart_ray_arrays(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("origin_x", "origin_y", "origin_z", "dir_x", "dir_y", "dir_z",
                                          "energy_keV", "pol_x", "pol_y", "pol_z")]


class heart_tally(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("emitted", "miss", "absorbed", "exit_front", "exit_back",
                                          "exit_side", "capped", "stuck", "no_bragg", "det_hits")] + \
               [("refl_hist", C.c_uint64 * 16), ("collisions", C.c_uint64)]

    def as_dict(self):
        d = {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "refl_hist"}
        d["refl_hist"] = [int(x) for x in self.refl_hist]
        return d


class heart_qe_table(C.Structure):
    _fields_ = [("keV", C.POINTER(C.c_double)), ("qe", C.POINTER(C.c_double)), ("n", C.c_int32),
                ("reserved", C.c_int32)]


def make_qe(table):
    """[(keV, qe), ...] -> heart_qe_table (keeps its arrays alive); None for no table"""
    if not table:
        return None
    e = (C.c_double * len(table))(*[float(a) for a, _ in table])
    q = (C.c_double * len(table))(*[float(b) for _, b in table])
    t = heart_qe_table()
    t.keV = e
    t.qe = q
    t.n = len(table)
    t._keep = (e, q)
    return t


class heart_tune(C.Structure):
    _fields_ = [("blocks_per_sm", C.c_int32), ("refill_lanes", C.c_int32), ("max_chunk_rays", C.c_uint32),
                ("reserved", C.c_int32), ("rays_per_s", C.c_double)]


PIPE_OPS = ["ffma", "lop3", "iadd3", "imad", "imad_hi", "imad_wide", "mufu_rsq", "mufu_ex2", "mufu_lg2", "dfma"]


class heart_pipe_rates(C.Structure):
    _fields_ = [("warp_inst_per_s", C.c_double * len(PIPE_OPS)),
                ("warp_inst_per_clk_sm", C.c_double * len(PIPE_OPS)),
                ("sm_clock_hz", C.c_double), ("sms", C.c_int32), ("n_ops", C.c_int32)]


RECORD_DTYPE = np.dtype([
    ("ray_id", np.uint64), ("outcome", np.int32), ("nrefl", np.int32), ("ncoll", np.int64),
    ("energy_keV", np.float64), ("pos", np.float64, 3), ("dir", np.float64, 3),
    ("u_mm", np.float64), ("v_mm", np.float64), ("ix", np.int32), ("iy", np.int32),
    ("det_hit", np.int32), ("no_bragg", np.int32), ("pol", np.float64, 3)])
assert RECORD_DTYPE.itemsize == 136

EXPORTS = ["heart_spectrometer_create", "heart_spectrometer_destroy", "heart_trace", "heart_trace_energy",
           "heart_trace_host", "heart_trace_rays",
           "heart_trace_records", "heart_trace_batch", "heart_trace_batch_static", "heart_autotune", "heart_server_create", "heart_server_destroy",
           "heart_submit", "heart_poll", "heart_release", "heart_fetch_image", "heart_job_latency",
           "heart_pipe_peaks", "heart_calibration_map", "heart_check_functions", "heart_last_error"]


class HeartError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None


def library(path=None):
    """Load libheart.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libheart.so is not built (%s); run __graft_entry__.build()" % p)
    L = C.CDLL(p)
    vp, u64, i32 = C.c_void_p, C.c_uint64, C.c_int32
    L.heart_spectrometer_create.argtypes = [C.POINTER(heart_spectrometer_desc), C.POINTER(vp)]
    L.heart_spectrometer_destroy.argtypes = [vp]
    L.heart_trace.argtypes = [vp, C.POINTER(heart_source_desc), u64, u64, u64, vp, i32, vp,
                              C.POINTER(heart_tally)]
    L.heart_trace_host.argtypes = [vp, C.POINTER(heart_source_desc), u64, u64, u64, vp, i32,
                                   C.POINTER(heart_tally)]
    L.heart_trace_energy.argtypes = [vp, C.POINTER(heart_source_desc), u64, u64, u64, vp, vp,
                                     C.POINTER(heart_qe_table), i32, vp, C.POINTER(heart_tally)]
    L.heart_trace_records.argtypes = [vp, C.POINTER(heart_source_desc), u64, u64, u64, vp, i32, vp, vp,
                                      C.POINTER(heart_tally)]
    L.heart_trace_rays.argtypes = [vp, C.POINTER(heart_ray_arrays), u64, u64, u64, vp, i32, vp, vp,
                                   C.POINTER(heart_tally)]
    L.heart_trace_batch.argtypes = [C.POINTER(vp), C.POINTER(C.POINTER(heart_source_desc)),
                                    C.POINTER(u64), C.POINTER(u64), C.POINTER(vp), i32, vp,
                                    C.POINTER(heart_tally)]
    L.heart_trace_batch_static.argtypes = L.heart_trace_batch.argtypes
    L.heart_autotune.argtypes = [vp, C.POINTER(heart_source_desc), u64, vp, C.POINTER(heart_tune)]
    L.heart_server_create.argtypes = [C.c_size_t, C.POINTER(vp)]
    L.heart_server_destroy.argtypes = [vp]
    L.heart_submit.argtypes = [vp, vp, C.POINTER(heart_source_desc), u64, u64, i32, C.POINTER(u64)]
    L.heart_poll.argtypes = [vp, u64, i32, C.POINTER(heart_tally), C.POINTER(vp)]
    L.heart_release.argtypes = [vp, u64]
    L.heart_job_latency.argtypes = [vp, u64, C.POINTER(C.c_double)]
    L.heart_fetch_image.argtypes = [vp, u64, vp, i32]
    L.heart_pipe_peaks.argtypes = [vp, C.POINTER(heart_pipe_rates)]
    L.heart_check_functions.argtypes = [vp, i32, vp, vp, vp, vp, u64, vp]
    L.heart_calibration_map.argtypes = [vp, C.POINTER(heart_source_desc), C.c_double, C.c_double, u64, u64, i32,
                                        vp, vp, vp, vp, C.POINTER(heart_tally)]
    L.heart_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name != "heart_last_error":
            getattr(L, name).restype = C.c_int
    if path is None:
        _lib = L
    return L


def _check(status, allow=(0,)):
    if status not in allow:
        raise HeartError(status, library().heart_last_error().decode())
    return status


def make_desc(d):
    """Neutral parameter dict (see workloads.py) -> heart_spectrometer_desc."""
    s = heart_spectrometer_desc()
    s.d_spacing_A = d["d_spacing_A"]
    s.thickness_mm = d["thickness_mm"]
    s.geometry = GEOMETRY[d["geometry"]]
    s.mdf = MDF[d["mdf"]]
    s.radius_mm = d.get("radius_mm", 0.0)
    s.centre_mm = D3(*d["centre_mm"])
    s.normal = D3(*d["normal"])
    s.axis = D3(*d["axis"])
    s.centre_axial_mm = d.get("centre_axial_mm", 0.0)
    s.size_disp_mm = d["size_disp_mm"]
    s.size_nondisp_mm = d["size_nondisp_mm"]
    s.mdf_fwhm_rad = d["mdf_fwhm_rad"]
    s.mdf_eta = d.get("mdf_eta", 0.0)
    s.irc = IRC[d["irc"]]
    s.max_reflections = d["max_reflections"]
    s.irc_fwhm_rad = d["irc_fwhm_rad"]
    s.irc_lorentz_fwhm_rad = d.get("irc_lorentz_fwhm_rad", 0.0)
    s.irc_shift_rad = d.get("irc_shift_rad", 0.0)
    s.prins_g = d.get("prins_g", 0.0)
    s.absorption_length_mm = d["absorption_length_mm"]
    s.absorption_ref_keV = d.get("absorption_ref_keV", 8.0)
    s.absorption_power = d.get("absorption_power", 0.0)
    s.refl_K_per_mm2 = d.get("refl_K_per_mm2", -1.0)
    s.refl_darwin_fwhm_rad = d.get("refl_darwin_fwhm_rad", d["irc_fwhm_rad"])
    s.refl_ref_keV = d.get("refl_ref_keV", 8.0)
    s.max_collisions = d.get("max_collisions", 1_000_000)
    s.det_centre_mm = D3(*d["det_centre_mm"])
    s.det_u = D3(*d["det_u"])
    s.det_v = D3(*d["det_v"])
    s.det_nx = d["det_nx"]
    s.det_ny = d["det_ny"]
    s.pixel_mm = d["pixel_mm"]
    s.count_type = COUNT[d.get("count_type", "i32")]
    s.sampler = SAMPLER[d.get("sampler", "thinned")]
    s.thin_vstar = d.get("thin_vstar", 0.0)
    # reflection orders: (multiple m, K ratio, width ratio) each; absent: the single reflection
    orders = d.get("orders") or []
    if len(orders) > 4:
        raise ValueError("at most 4 reflection orders")
    s.n_orders = len(orders)
    for h, (m, kr, wr) in enumerate(orders):
        s.order_m[h], s.order_K_rel[h], s.order_w_rel[h] = int(m), kr, wr
    # energy-dependent rocking curve: (keV, width scale, added shift rad) knots
    knots = d.get("irc_energy") or []
    if len(knots) > 16:
        raise ValueError("at most 16 rocking-curve energy knots")
    s.n_irc_e = len(knots)
    for i, (e, ws, sh) in enumerate(knots):
        s.irc_e_keV[i], s.irc_e_wscale[i], s.irc_e_shift_rad[i] = e, ws, sh
    return s


def make_source(d):
    """Neutral source dict -> heart_source_desc (keeps its component array alive)."""
    comps = d["components"]
    arr = (heart_spectral_component * len(comps))()
    for i, c in enumerate(comps):
        arr[i].kind = SRC[c["kind"]]
        arr[i].e0_keV = c.get("e0_keV", 0.0)
        arr[i].width_keV = c.get("width_keV", 0.0)
        arr[i].lo_keV = c.get("lo_keV", 0.0)
        arr[i].hi_keV = c.get("hi_keV", 0.0)
        arr[i].weight = c.get("weight", 1.0)
    s = heart_source_desc()
    s.components = arr
    s.n_components = len(comps)
    s.origin_mm = D3(*d["origin_mm"])
    s.axis = D3(*d["axis"])
    s.cone_half_angle_rad = d["cone_half_angle_rad"]
    s.spot_fwhm_mm = (C.c_double * 2)(*d.get("spot_fwhm_mm", (0.0, 0.0)))
    s.polarization = D3(*d.get("polarization", (0.0, 0.0, 0.0)))
    keep = [arr]
    if d.get("table") is not None:
        keV = np.ascontiguousarray(np.asarray(d["table"][0], dtype=np.float64))
        pdf = np.ascontiguousarray(np.asarray(d["table"][1], dtype=np.float64))
        s.table_keV = keV.ctypes.data_as(C.POINTER(C.c_double))
        s.table_pdf = pdf.ctypes.data_as(C.POINTER(C.c_double))
        s.n_table = min(len(keV), len(pdf))
        keep += [keV, pdf]
    s._keep = keep
    return s


class Spectrometer:
    """Owns a heart_spectrometer handle (device tables)."""

    def __init__(self, desc_dict):
        self.desc = dict(desc_dict)
        self._c = make_desc(desc_dict)
        h = C.c_void_p()
        _check(library().heart_spectrometer_create(C.byref(self._c), C.byref(h)))
        self.handle = h
        self.shape = (desc_dict["det_ny"], desc_dict["det_nx"])
        self.count_dtype = "int64" if desc_dict.get("count_type", "i32") == "i64" else "int32"

    def close(self):
        if self.handle is not None and self.handle.value:
            library().heart_spectrometer_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def heart_spectrometer_create(desc_dict):
    return Spectrometer(desc_dict)


def heart_spectrometer_destroy(spec):
    spec.close()


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def heart_trace(spec, source, n_rays, seed, ray_offset, d_image, precision="fp32", stream=None,
                want_tally=True):
    """Trace on the device; d_image is a CUDA tensor (+= counts)."""
    src = make_source(source)
    t = heart_tally()
    st = library().heart_trace(spec.handle, C.byref(src), int(n_rays), int(seed), int(ray_offset),
                               C.c_void_p(d_image.data_ptr()), PRECISION[precision],
                               C.c_void_p(_stream_ptr(stream)), C.byref(t) if want_tally else None)
    _check(st, allow=(0, 6))
    return t.as_dict() if want_tally else None


def heart_trace_energy(spec, source, n_rays, seed, ray_offset, d_image, d_energy, qe=None, precision="fp32",
                       stream=None):
    """Counts into d_image (may be None) and energy x QE (uint64 / int64 CUDA
    tensor, units of 1e-6 keV) into d_energy.  qe: [(keV, qe), ...] or None."""
    src = make_source(source)
    q = make_qe(qe)
    t = heart_tally()
    st = library().heart_trace_energy(spec.handle, C.byref(src), int(n_rays), int(seed), int(ray_offset),
                                      C.c_void_p(d_image.data_ptr()) if d_image is not None else None,
                                      C.c_void_p(d_energy.data_ptr()), C.byref(q) if q is not None else None,
                                      PRECISION[precision], C.c_void_p(_stream_ptr(stream)), C.byref(t))
    _check(st, allow=(0, 6))
    return t.as_dict()


def heart_calibration_map(spec, source, min_keV, max_keV, n_rays, seed, precision="fp32", stream=None):
    """Energy dispersion of the detector (Sec. 3): the source geometry with a
    uniform spectrum on [min_keV, max_keV]; returns (mean keV per pixel as a
    float64 CUDA tensor, NaN where no photon landed; count image; tallies).
    The division runs in the library (heart_calibration_map)."""
    import torch
    src = make_source(source)
    counts = torch.zeros(spec.shape, dtype=torch.int64 if spec.count_dtype == "int64" else torch.int32,
                         device="cuda")
    energy = torch.zeros(spec.shape, dtype=torch.int64, device="cuda")
    mean = torch.empty(spec.shape, dtype=torch.float64, device="cuda")
    t = heart_tally()
    st = library().heart_calibration_map(spec.handle, C.byref(src), float(min_keV), float(max_keV), int(n_rays),
                                         int(seed), PRECISION[precision], C.c_void_p(counts.data_ptr()),
                                         C.c_void_p(energy.data_ptr()), C.c_void_p(mean.data_ptr()),
                                         C.c_void_p(_stream_ptr(stream)), C.byref(t))
    _check(st, allow=(0, 6))
    return mean, counts, t.as_dict()


def calibration_map(spec, source, min_keV, max_keV, n_rays, seed, precision="fp32", stream=None):
    """(mean keV per pixel, count image) of heart_calibration_map"""
    mean, counts, _ = heart_calibration_map(spec, source, min_keV, max_keV, n_rays, seed, precision, stream)
    return mean, counts


def heart_trace_host(spec, source, n_rays, seed, ray_offset, h_image, precision="fp32"):
    """Host-memory variant: h_image (numpy, C-contiguous, += counts)."""
    src = make_source(source)
    t = heart_tally()
    assert h_image.flags["C_CONTIGUOUS"]
    st = library().heart_trace_host(spec.handle, C.byref(src), int(n_rays), int(seed), int(ray_offset),
                                    C.c_void_p(h_image.ctypes.data), PRECISION[precision], C.byref(t))
    _check(st, allow=(0, 6))
    return t.as_dict()


def heart_trace_records(spec, source, n_rays, seed, ray_offset=0, precision="fp64", d_image=None, stream=None,
                        on_device=False):
    """Per-ray records (numpy structured array) and tallies.  on_device: return
    the records as a CUDA uint8 tensor instead (decode slices with
    records_from_device), for traces too large to copy whole."""
    import torch
    src = make_source(source)
    t = heart_tally()
    rec = torch.empty(int(n_rays) * RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    st = library().heart_trace_records(spec.handle, C.byref(src), int(n_rays), int(seed), int(ray_offset),
                                       C.c_void_p(d_image.data_ptr()) if d_image is not None else None,
                                       PRECISION[precision], C.c_void_p(rec.data_ptr()),
                                       C.c_void_p(_stream_ptr(stream)), C.byref(t))
    _check(st, allow=(0, 6))
    if on_device:
        return rec, t.as_dict()
    out = np.frombuffer(rec.cpu().numpy().tobytes(), dtype=RECORD_DTYPE)
    return out, t.as_dict()


def records_from_device(rec, first, count):
    """records first .. first + count - 1 of a device record tensor (heart_trace_records(on_device=True))"""
    b = RECORD_DTYPE.itemsize
    return np.frombuffer(rec[first * b:(first + count) * b].cpu().numpy().tobytes(), dtype=RECORD_DTYPE)


def heart_trace_rays(spec, rays, seed, ray_offset, d_image, precision="fp32", records=False, stream=None):
    """Trace user-supplied rays.  `rays` maps origin_x ... energy_keV (and
    optionally pol_x, pol_y, pol_z) to contiguous float64 CUDA tensors of one
    length.  Returns the tallies, and the per-ray records if asked for."""
    import torch
    names = [f for f, _ in heart_ray_arrays._fields_]
    keep = {}
    ra = heart_ray_arrays()
    n = None
    for f in names:
        t = rays.get(f)
        if t is None:
            continue
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{f}: contiguous float64 CUDA tensor expected")
        if n is None:
            n = t.numel()
        if t.numel() != n:
            raise ValueError("ray arrays differ in length")
        keep[f] = t
        setattr(ra, f, t.data_ptr())
    n = 0 if n is None else n
    t = heart_tally()
    rec = None
    if records:
        rec = torch.empty(max(n, 1) * RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    st = library().heart_trace_rays(spec.handle, C.byref(ra), int(n), int(seed), int(ray_offset),
                                    C.c_void_p(d_image.data_ptr()) if d_image is not None else None,
                                    PRECISION[precision], C.c_void_p(rec.data_ptr()) if rec is not None else None,
                                    C.c_void_p(_stream_ptr(stream)), C.byref(t))
    _check(st, allow=(0, 6))
    if records:
        out = np.frombuffer(rec.cpu().numpy().tobytes(), dtype=RECORD_DTYPE)[:n]
        return out, t.as_dict()
    return t.as_dict()


def heart_trace_batch(specs, sources, n_rays, seeds, d_images, stream=None):
    """Many spectrometers, FP32: jobs below 2^18 rays in one persistent launch,
    larger ones as two-pass traces (each equal to its single heart_trace)."""
    n = len(specs)
    srcs = [make_source(s) for s in sources]
    hs = (C.c_void_p * n)(*[s.handle.value for s in specs])
    sp = (C.POINTER(heart_source_desc) * n)(*[C.pointer(s) for s in srcs])
    nr = (C.c_uint64 * n)(*[int(x) for x in n_rays])
    sd = (C.c_uint64 * n)(*[int(x) for x in seeds])
    im = (C.c_void_p * n)(*[d.data_ptr() for d in d_images])
    tl = (heart_tally * n)()
    st = library().heart_trace_batch(hs, sp, nr, sd, im, n, C.c_void_p(_stream_ptr(stream)), tl)
    _check(st, allow=(0, 6))
    return [tl[i].as_dict() for i in range(n)]


STATIC_MAX_JOBS = 64


CHECK_FUNCTIONS = {"acos_ratio": 0, "irc_rel": 1, "irc_bound": 2, "arc_bound": 3, "arc_measure": 4}


def heart_check_functions(spec, which, x, y=None, z=None):
    """a device function of the FP32 kernels on float32 CUDA tensors (tests)"""
    import torch
    x = x.contiguous()
    y = y.contiguous() if y is not None else None
    z = z.contiguous() if z is not None else None
    out = torch.empty_like(x)
    st = library().heart_check_functions(spec.handle if spec is not None else None, CHECK_FUNCTIONS[which],
                                         C.c_void_p(x.data_ptr()),
                                         C.c_void_p(y.data_ptr()) if y is not None else None,
                                         C.c_void_p(z.data_ptr()) if z is not None else None,
                                         C.c_void_p(out.data_ptr()), x.numel(),
                                         C.c_void_p(_stream_ptr(None)))
    _check(st)
    torch.cuda.synchronize()
    return out


def heart_pipe_peaks(stream=None):
    """Issue rates of the FP32, integer, SFU and FP64 pipes on this GPU (one
    microbenchmark kernel per instruction): {op: (warp instructions per second,
    warp instructions per SM per clock)} plus the SM clock and SM count."""
    r = heart_pipe_rates()
    _check(library().heart_pipe_peaks(C.c_void_p(_stream_ptr(stream)), C.byref(r)))
    out = {op: (r.warp_inst_per_s[i], r.warp_inst_per_clk_sm[i]) for i, op in enumerate(PIPE_OPS)}
    out["sm_clock_hz"] = r.sm_clock_hz
    out["sms"] = r.sms
    return out


def heart_autotune(spec, source, probe_rays=1 << 24, stream=None):
    """Pick the FP32 launch shape (blocks per SM, refill threshold) by timing
    probes; the choice applies to every later FP32 launch of the process."""
    src = make_source(source)
    t = heart_tune()
    _check(library().heart_autotune(spec.handle, C.byref(src), int(probe_rays),
                                    C.c_void_p(_stream_ptr(stream)), C.byref(t)))
    return {"blocks_per_sm": t.blocks_per_sm, "refill_lanes": t.refill_lanes,
            "max_chunk_rays": t.max_chunk_rays, "probe_rays_per_s": t.rays_per_s}


def heart_trace_batch_static(specs, sources, n_rays, seeds, d_images, stream=None):
    """As heart_trace_batch, on the library's fixed device work area: the call
    allocates no device memory (for callers that cannot allocate while they
    run).  At most STATIC_MAX_JOBS jobs; calls share the work area, so
    serialise them."""
    n = len(specs)
    srcs = [make_source(s) for s in sources]
    hs = (C.c_void_p * n)(*[s.handle.value for s in specs])
    sp = (C.POINTER(heart_source_desc) * n)(*[C.pointer(s) for s in srcs])
    nr = (C.c_uint64 * n)(*[int(x) for x in n_rays])
    sd = (C.c_uint64 * n)(*[int(x) for x in seeds])
    im = (C.c_void_p * n)(*[d.data_ptr() for d in d_images])
    tl = (heart_tally * max(n, 1))()
    st = library().heart_trace_batch_static(hs, sp, nr, sd, im, n, C.c_void_p(_stream_ptr(stream)), tl)
    _check(st, allow=(0, 6))
    return [tl[i].as_dict() for i in range(n)]


class Server:
    def __init__(self, mem_cap_bytes):
        h = C.c_void_p()
        _check(library().heart_server_create(int(mem_cap_bytes), C.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, spec, source, n_rays, seed, precision="fp32"):
        src = make_source(source)
        jid = C.c_uint64()
        _check(library().heart_submit(self.handle, spec.handle, C.byref(src), int(n_rays), int(seed),
                                      PRECISION[precision], C.byref(jid)))
        self._keep[jid.value] = spec
        return jid.value

    def poll(self, job_id, timeout_ms=0):
        """(status_name, tally or None, device image pointer or None)."""
        t = heart_tally()
        img = C.c_void_p()
        st = library().heart_poll(self.handle, int(job_id), int(timeout_ms), C.byref(t), C.byref(img))
        if st in (4, 5):
            return STATUS[st], None, None
        _check(st, allow=(0, 6))
        return STATUS[st], t.as_dict(), img.value

    def fetch(self, job_id, out):
        """copy the finished job's image into `out` (CUDA tensor or numpy array)"""
        if hasattr(out, "data_ptr"):
            ptr, host = out.data_ptr(), int(not out.is_cuda)
        else:
            ptr, host = out.ctypes.data, 1
        _check(library().heart_fetch_image(self.handle, int(job_id), C.c_void_p(ptr), host))
        return out

    def latency(self, job_id):
        """server-measured seconds from submit to completion"""
        v = C.c_double()
        _check(library().heart_job_latency(self.handle, int(job_id), C.byref(v)))
        return v.value

    def release(self, job_id):
        _check(library().heart_release(self.handle, int(job_id)))
        self._keep.pop(job_id, None)

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(library().heart_server_destroy(self.handle))
        self.handle = None


def heart_server_create(mem_cap_bytes):
    return Server(mem_cap_bytes)


def heart_submit(server, spec, source, n_rays, seed, precision="fp32"):
    return server.submit(spec, source, n_rays, seed, precision)


def heart_poll(server, job_id, timeout_ms=0):
    return server.poll(job_id, timeout_ms)


def heart_release(server, job_id):
    return server.release(job_id)


def heart_server_destroy(server):
    server.close()
