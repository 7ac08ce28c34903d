"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
arm import this module.  It converts the neutral parameter dictionaries of
paper_2503_16955_gb300.workloads into the oracle's own C structures and calls
liboracle.so; it shares no code with the product's binding.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

GEOMETRY = {"flat": 0, "cyl": 1}
MDF = {"gaussian": 0, "lorentzian": 1, "pseudo_voigt": 2, "vmf": 3, "wl": 4, "swl": 5, "uniform": 6}
IRC = {"darwin": 0, "darwin_prins": 1, "pseudo_voigt": 2, "gaussian": 3, "lorentzian": 4, "box": 5,
       "none": 6}
SRC = {"mono": 0, "gauss": 1, "lorentz": 2, "inv_e": 3, "uniform": 4, "table": 5}
OUTCOME = {0: "miss", 1: "absorbed", 2: "exit_front", 3: "exit_back", 4: "exit_side",
           5: "capped", 6: "stuck"}
MDF_M = 4096
MDF_T = 256
MAX_COMP = 16

D3 = C.c_double * 3


class Spec(C.Structure):
    _fields_ = [
        ("d_spacing_A", C.c_double), ("thickness_mm", C.c_double),
        ("geometry", C.c_int32), ("mdf", C.c_int32),
        ("radius_mm", C.c_double),
        ("centre", D3), ("normal", D3), ("axis", D3),
        ("centre_axial_mm", C.c_double),
        ("size_disp_mm", C.c_double), ("size_nondisp_mm", C.c_double),
        ("mdf_fwhm_rad", C.c_double), ("mdf_eta", C.c_double),
        ("irc", C.c_int32), ("max_reflections", C.c_int32),
        ("irc_fwhm_rad", C.c_double), ("irc_lorentz_fwhm_rad", C.c_double),
        ("irc_shift_rad", C.c_double), ("prins_g", C.c_double),
        ("absorption_length_mm", C.c_double), ("absorption_ref_keV", C.c_double),
        ("absorption_power", C.c_double),
        ("refl_K_per_mm2", C.c_double), ("refl_darwin_fwhm_rad", C.c_double),
        ("refl_ref_keV", C.c_double),
        ("max_collisions", C.c_int64),
        ("det_centre", D3), ("det_u", D3), ("det_v", D3),
        ("det_nx", C.c_int32), ("det_ny", C.c_int32),
        ("pixel_mm", C.c_double),
        ("sampler", C.c_int32), ("pad3", C.c_int32), ("thin_vstar", C.c_double),
        ("n_orders", C.c_int32), ("pad4", C.c_int32), ("order_m", C.c_int32 * 4),
        ("order_K_rel", C.c_double * 4), ("order_w_rel", C.c_double * 4),
        ("n_irc_e", C.c_int32), ("pad5", C.c_int32), ("irc_e_keV", C.c_double * 16),
        ("irc_e_wscale", C.c_double * 16), ("irc_e_shift_rad", C.c_double * 16),
    ]

SAMPLER = {"plain": 0, "thinned": 1}


class Component(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("e0_keV", C.c_double),
                ("width_keV", C.c_double), ("lo_keV", C.c_double), ("hi_keV", C.c_double),
                ("weight", C.c_double)]


class Source(C.Structure):
    _fields_ = [("n_comp", C.c_int32), ("pad", C.c_int32), ("comp", Component * MAX_COMP),
                ("origin", D3), ("axis", D3), ("cone_half_angle_rad", C.c_double),
                ("spot_fwhm_mm", C.c_double * 2), ("polarization", D3),
                ("table_keV", C.POINTER(C.c_double)), ("table_pdf", C.POINTER(C.c_double)),
                ("n_table", C.c_int32), ("pad2", C.c_int32)]


class Rays(C.Structure):
    _fields_ = [(n, C.POINTER(C.c_double)) for n in ("ox", "oy", "oz", "kx", "ky", "kz", "E", "px", "py", "pz")]


class Tally(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("emitted", "miss", "absorbed", "exit_front", "exit_back",
                                          "exit_side", "capped", "stuck", "no_bragg", "det_hits")] + \
               [("refl_hist", C.c_uint64 * 16), ("collisions", C.c_uint64)]

    def as_dict(self):
        d = {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "refl_hist"}
        d["refl_hist"] = [int(x) for x in self.refl_hist]
        return d


RECORD_DTYPE = np.dtype([
    ("ray_id", np.uint64), ("outcome", np.int32), ("nrefl", np.int32), ("ncoll", np.int64),
    ("energy_keV", np.float64), ("pos", np.float64, 3), ("dir", np.float64, 3),
    ("u_mm", np.float64), ("v_mm", np.float64), ("ix", np.int32), ("iy", np.int32),
    ("det_hit", np.int32), ("no_bragg", np.int32), ("pol", np.float64, 3)])


class RayConsts(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E_keV", "lambda_A", "sin_aB", "alpha_B", "mu0", "Q",
                                          "mubar", "p_abs")] + [("no_bragg", C.c_int32),
                                                                ("pad", C.c_int32),
                                                                ("n_orders", C.c_int32), ("pad2", C.c_int32),
                                                                ("shift_rad", C.c_double)] + \
        [(n, C.c_double * 4) for n in ("ord_sin", "ord_alpha", "ord_Q", "ord_w", "ord_qr")]


class QE(C.Structure):
    _fields_ = [("n", C.c_int32), ("pad", C.c_int32), ("keV", C.c_double * 32), ("qe", C.c_double * 32)]


def make_qe(table):
    """[(keV, qe), ...] -> QE (None / empty: QE = 1)"""
    q = QE()
    table = list(table or [])
    if len(table) > 32:
        raise ValueError("at most 32 QE knots")
    q.n = len(table)
    for i, (e, v) in enumerate(table):
        q.keV[i] = e
        q.qe[i] = v
    return q


class MdfTable(C.Structure):
    _fields_ = [("body", C.c_double * MDF_M), ("tail", C.c_double * (MDF_T + 1)), ("qmax", C.c_double)]


class SegInfo(C.Structure):
    _fields_ = [("s_exit", C.c_double), ("face", C.c_int32), ("thinned", C.c_int32),
                ("kN0", C.c_double), ("kN1", C.c_double), ("xstar", C.c_double), ("vstar", C.c_double),
                ("irc_max", C.c_double), ("W0", C.c_double), ("none_qv", C.c_double), ("alpha0", C.c_double),
                ("ra", C.c_double), ("qmin", C.c_double), ("pbar", C.c_double), ("S1", C.c_double),
                ("S2", C.c_double), ("w0", C.c_uint64), ("wspan", C.c_uint64), ("lam", C.c_double),
                ("mu", C.c_double), ("pa", C.c_double), ("wn", C.c_double), ("wf", C.c_double),
                ("psis", C.c_double), ("pin", C.c_double), ("pio", C.c_double), ("w1", C.c_uint64),
                ("w2", C.c_uint64), ("pbarB", C.c_double), ("sA", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp, u32p, i64p = C.POINTER(C.c_double), C.POINTER(C.c_uint32), C.POINTER(C.c_int64)
        sig = {
            "orc_philox4x32_10": (None, [u32p, u32p, u32p]),
            "orc_pv_width": (None, [C.c_double, C.c_double, dp, dp]),
            "orc_irc": (C.c_double, [C.POINTER(Spec), C.c_double]),
            "orc_irc_max": (C.c_double, [C.POINTER(Spec)]),
            "orc_darwin_prins_area": (C.c_double, [C.c_double]),
            "orc_mdf_W": (C.c_double, [C.POINTER(Spec), C.c_double]),
            "orc_mdf_qmax": (C.c_double, [C.POINTER(Spec)]),
            "orc_mdf_norm": (C.c_double, [C.POINTER(Spec)]),
            "orc_mdf_cdf": (C.c_double, [C.POINTER(Spec), C.c_double]),
            "orc_mdf_ccdf": (C.c_double, [C.POINTER(Spec), C.c_double]),
            "orc_mdf_quantile_exact": (C.c_double, [C.POINTER(Spec), C.c_double, C.c_int, C.c_double]),
            "orc_mdf_build_table": (C.c_int, [C.POINTER(Spec), C.POINTER(MdfTable)]),
            "orc_mdf_table_lookup": (C.c_double, [C.POINTER(MdfTable), C.c_uint32]),
            "orc_ray_constants": (C.c_int, [C.POINTER(Spec), C.c_double, C.POINTER(RayConsts)]),
            "orc_trace": (C.c_int, [C.POINTER(Spec), C.POINTER(Source), C.c_uint64, C.c_uint64,
                                    C.c_uint64, C.c_int, i64p, C.POINTER(Tally), C.c_void_p]),
            "orc_trace_energy": (C.c_int, [C.POINTER(Spec), C.POINTER(Source), C.c_uint64, C.c_uint64,
                                           C.c_uint64, C.c_int, i64p, i64p, C.POINTER(QE), C.POINTER(Tally),
                                           C.c_void_p]),
            "orc_qe_eval": (C.c_double, [C.POINTER(QE), C.c_double]),
            "orc_trace_rays": (C.c_int, [C.POINTER(Spec), C.POINTER(Rays), C.c_uint64, C.c_uint64, C.c_uint64,
                                         C.c_int, i64p, i64p, C.POINTER(QE), C.POINTER(Tally), C.c_void_p]),
            "orc_walk_injected": (C.c_int, [C.POINTER(Spec), C.c_double, dp, dp, dp, u32p, C.c_int64,
                                            C.c_void_p]),
            "orc_walk_injected_n": (C.c_int, [C.POINTER(Spec), C.c_int64, dp, dp, dp, dp, u32p, C.c_int64,
                                              C.c_void_p]),
            "orc_sample_crystallites": (C.c_int64, [C.POINTER(Spec), C.c_double, C.c_double,
                                                    C.c_int64, C.c_uint64, dp, dp]),
            "orc_reflection_rate": (C.c_double, [C.POINTER(Spec), C.c_double, C.c_double]),
            "orc_segment_bounds": (C.c_int, [C.POINTER(Spec), C.c_int64, dp, dp, dp, C.c_int, C.POINTER(SegInfo)]),
            "orc_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _err():
    return lib().orc_last_error().decode()


def make_spec(d):
    """Neutral dict -> oracle Spec."""
    s = Spec()
    s.d_spacing_A = d["d_spacing_A"]
    s.thickness_mm = d["thickness_mm"]
    s.geometry = GEOMETRY[d["geometry"]]
    s.mdf = MDF[d["mdf"]]
    s.radius_mm = d.get("radius_mm", 0.0)
    s.centre = D3(*d["centre_mm"])
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
    s.det_centre = D3(*d["det_centre_mm"])
    s.det_u = D3(*d["det_u"])
    s.det_v = D3(*d["det_v"])
    s.det_nx = d["det_nx"]
    s.det_ny = d["det_ny"]
    s.pixel_mm = d["pixel_mm"]
    s.sampler = SAMPLER[d.get("sampler", "thinned")]
    s.thin_vstar = d.get("thin_vstar", 0.0)
    # reflection orders: list of (multiple m, K ratio, width ratio); absent: the single reflection
    orders = d.get("orders") or []
    s.n_orders = len(orders)
    for h, (m, kr, wr) in enumerate(orders[:4]):
        s.order_m[h] = int(m)
        s.order_K_rel[h] = kr
        s.order_w_rel[h] = wr
    # energy-dependent rocking curve: list of (keV, width scale, added shift rad)
    knots = d.get("irc_energy") or []
    s.n_irc_e = len(knots)
    for i, (e, ws, sh) in enumerate(knots[:16]):
        s.irc_e_keV[i] = e
        s.irc_e_wscale[i] = ws
        s.irc_e_shift_rad[i] = sh
    return s


def make_source(d):
    s = Source()
    comps = d["components"]
    if not 1 <= len(comps) <= MAX_COMP:
        raise ValueError("1..16 spectral components")
    s.n_comp = len(comps)
    for i, c in enumerate(comps):
        s.comp[i].kind = SRC[c["kind"]]
        s.comp[i].e0_keV = c.get("e0_keV", 0.0)
        s.comp[i].width_keV = c.get("width_keV", 0.0)
        s.comp[i].lo_keV = c.get("lo_keV", 0.0)
        s.comp[i].hi_keV = c.get("hi_keV", 0.0)
        s.comp[i].weight = c.get("weight", 1.0)
    s.origin = D3(*d["origin_mm"])
    s.axis = D3(*d["axis"])
    s.cone_half_angle_rad = d["cone_half_angle_rad"]
    sf = d.get("spot_fwhm_mm", (0.0, 0.0))
    s.spot_fwhm_mm = (C.c_double * 2)(*sf)
    s.polarization = D3(*d.get("polarization", (0.0, 0.0, 0.0)))
    if d.get("table") is not None:
        keV = np.ascontiguousarray(np.asarray(d["table"][0], dtype=np.float64))
        pdf = np.ascontiguousarray(np.asarray(d["table"][1], dtype=np.float64))
        s.table_keV = keV.ctypes.data_as(C.POINTER(C.c_double))
        s.table_pdf = pdf.ctypes.data_as(C.POINTER(C.c_double))
        s.n_table = min(len(keV), len(pdf))
        s._keep = (keV, pdf)
    return s


def philox(counter, key):
    ctr = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in counter])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    out = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(ctr, k, out)
    return [int(x) for x in out]


def pv_width(fg, fl):
    F, eta = C.c_double(), C.c_double()
    lib().orc_pv_width(fg, fl, C.byref(F), C.byref(eta))
    return F.value, eta.value


def irc(spec_dict, x):
    s = make_spec(spec_dict)
    return np.array([lib().orc_irc(C.byref(s), float(v)) for v in np.atleast_1d(x)])


def irc_max(spec_dict):
    s = make_spec(spec_dict)
    return lib().orc_irc_max(C.byref(s))


def darwin_prins_area(g):
    return lib().orc_darwin_prins_area(g)


def mdf_W(spec_dict, q):
    s = make_spec(spec_dict)
    return np.array([lib().orc_mdf_W(C.byref(s), float(v)) for v in np.atleast_1d(q)])


def mdf_norm(spec_dict):
    s = make_spec(spec_dict)
    return lib().orc_mdf_norm(C.byref(s))


def mdf_qmax(spec_dict):
    s = make_spec(spec_dict)
    return lib().orc_mdf_qmax(C.byref(s))


def mdf_cdf(spec_dict, q):
    s = make_spec(spec_dict)
    return lib().orc_mdf_cdf(C.byref(s), q)


def mdf_ccdf(spec_dict, q):
    s = make_spec(spec_dict)
    return lib().orc_mdf_ccdf(C.byref(s), q)


def mdf_quantile_exact(spec_dict, u=0.0, comp=None):
    s = make_spec(spec_dict)
    if comp is not None:
        return lib().orc_mdf_quantile_exact(C.byref(s), 0.0, 1, comp)
    return lib().orc_mdf_quantile_exact(C.byref(s), u, 0, 0.0)


def mdf_table(spec_dict):
    s = make_spec(spec_dict)
    t = MdfTable()
    if lib().orc_mdf_build_table(C.byref(s), C.byref(t)) != 0:
        raise RuntimeError(_err())
    return t


def mdf_table_lookup(table, words):
    return np.array([lib().orc_mdf_table_lookup(C.byref(table), int(w)) for w in np.atleast_1d(words)])


def ray_constants(spec_dict, E):
    s = make_spec(spec_dict)
    c = RayConsts()
    lib().orc_ray_constants(C.byref(s), E, C.byref(c))
    out = {n: getattr(c, n) for n, _ in RayConsts._fields_ if not n.startswith("pad")}
    for n in ("ord_sin", "ord_alpha", "ord_Q", "ord_w", "ord_qr"):
        out[n] = [float(x) for x in out[n]][: c.n_orders]
    return out


def trace(spec_dict, source_dict, n_rays, seed, ray_offset=0, n_threads=0, records=False):
    """Trace n_rays; returns (int64 image [ny, nx], tally dict, records or None)."""
    s = make_spec(spec_dict)
    src = make_source(source_dict)
    img = np.zeros((spec_dict["det_ny"], spec_dict["det_nx"]), dtype=np.int64)
    tal = Tally()
    rec = np.zeros(n_rays, dtype=RECORD_DTYPE) if records else None
    rc = lib().orc_trace(C.byref(s), C.byref(src), n_rays, seed, ray_offset, n_threads,
                         img.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(tal),
                         rec.ctypes.data if records else None)
    if rc != 0:
        raise RuntimeError(_err())
    return img, tal.as_dict(), rec


def trace_energy(spec_dict, source_dict, n_rays, seed, qe=None, ray_offset=0, n_threads=0, records=False):
    """(count image, energy image in 1e-6 keV, tally, records)"""
    s = make_spec(spec_dict)
    src = make_source(source_dict)
    shape = (spec_dict["det_ny"], spec_dict["det_nx"])
    img = np.zeros(shape, dtype=np.int64)
    eimg = np.zeros(shape, dtype=np.int64)
    q = make_qe(qe)
    tal = Tally()
    rec = np.zeros(n_rays, dtype=RECORD_DTYPE) if records else None
    rc = lib().orc_trace_energy(C.byref(s), C.byref(src), n_rays, seed, ray_offset, n_threads,
                                img.ctypes.data_as(C.POINTER(C.c_int64)),
                                eimg.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(q), C.byref(tal),
                                rec.ctypes.data if records else None)
    if rc != 0:
        raise RuntimeError(_err())
    return img, eimg, tal.as_dict(), rec


def qe_eval(table, E):
    q = make_qe(table)
    return lib().orc_qe_eval(C.byref(q), E)


def trace_rays(spec_dict, rays, seed, qe=None, ray_offset=0, n_threads=0, records=False):
    """User-supplied rays: dict of float64 arrays ox, oy, oz, kx, ky, kz, E and
    optionally px, py, pz.  Returns (image, energy image, tally, records)."""
    s = make_spec(spec_dict)
    n = len(rays["E"])
    arrs = {k: np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for k, v in rays.items()}
    R = Rays()
    for k in ("ox", "oy", "oz", "kx", "ky", "kz", "E", "px", "py", "pz"):
        if k in arrs:
            setattr(R, k, arrs[k].ctypes.data_as(C.POINTER(C.c_double)))
    shape = (spec_dict["det_ny"], spec_dict["det_nx"])
    img = np.zeros(shape, dtype=np.int64)
    eimg = np.zeros(shape, dtype=np.int64)
    q = make_qe(qe)
    tal = Tally()
    rec = np.zeros(n, dtype=RECORD_DTYPE) if records else None
    rc = lib().orc_trace_rays(C.byref(s), C.byref(R), n, seed, ray_offset, n_threads,
                              img.ctypes.data_as(C.POINTER(C.c_int64)), eimg.ctypes.data_as(C.POINTER(C.c_int64)),
                              C.byref(q), C.byref(tal), rec.ctypes.data if records else None)
    if rc != 0:
        raise RuntimeError(_err())
    return img, eimg, tal.as_dict(), rec


def walk_injected(spec_dict, E, pos, direction, words, pol=None):
    s = make_spec(spec_dict)
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32))
    rec = np.zeros(1, dtype=RECORD_DTYPE)
    p = D3(*pos)
    d = D3(*direction)
    pp = D3(*pol) if pol is not None else None
    rc = lib().orc_walk_injected(C.byref(s), E, p, d, pp, w.ctypes.data_as(C.POINTER(C.c_uint32)),
                                 len(w), rec.ctypes.data)
    if rc != 0:
        raise RuntimeError(_err())
    return rec[0]


def walk_injected_n(spec_dict, E, pos, direction, words, pol=None):
    """many injected walks with one mosaic table: E (n,), pos/direction/pol
    (n, 3), words (n, m)"""
    s = make_spec(spec_dict)
    E = np.ascontiguousarray(np.asarray(E, dtype=np.float64))
    n = len(E)
    P = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(n, 3))
    D = np.ascontiguousarray(np.asarray(direction, dtype=np.float64).reshape(n, 3))
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32).reshape(n, -1))
    pp = None if pol is None else np.ascontiguousarray(np.asarray(pol, dtype=np.float64).reshape(n, 3))
    rec = np.zeros(n, dtype=RECORD_DTYPE)
    dp = C.POINTER(C.c_double)
    rc = lib().orc_walk_injected_n(C.byref(s), n, E.ctypes.data_as(dp), P.ctypes.data_as(dp), D.ctypes.data_as(dp),
                                   pp.ctypes.data_as(dp) if pp is not None else None,
                                   w.ctypes.data_as(C.POINTER(C.c_uint32)), w.shape[1], rec.ctypes.data)
    if rc != 0:
        raise RuntimeError(_err())
    return rec


def sample_crystallites(spec_dict, E, alpha, n, seed):
    s = make_spec(spec_dict)
    dl = np.zeros(n)
    ps = np.zeros(n)
    got = lib().orc_sample_crystallites(C.byref(s), E, alpha, n, seed,
                                        dl.ctypes.data_as(C.POINTER(C.c_double)),
                                        ps.ctypes.data_as(C.POINTER(C.c_double)))
    if got < 0:
        raise RuntimeError(_err())
    return dl[:got], ps[:got]


def reflection_rate(spec_dict, E, alpha):
    s = make_spec(spec_dict)
    return lib().orc_reflection_rate(C.byref(s), E, alpha)


def segment_bounds(spec_dict, E, pos, direction, order=0):
    """the thinned sampler's bounds of straight segments: E (n,), pos and
    direction (n, 3); returns a dict of arrays of the SegInfo fields"""
    s = make_spec(spec_dict)
    E = np.ascontiguousarray(np.atleast_1d(np.asarray(E, dtype=np.float64)))
    x = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    k = np.ascontiguousarray(np.asarray(direction, dtype=np.float64).reshape(-1, 3))
    n = len(E)
    out = (SegInfo * n)()
    dp = C.POINTER(C.c_double)
    if lib().orc_segment_bounds(C.byref(s), n, E.ctypes.data_as(dp), x.ctypes.data_as(dp),
                                k.ctypes.data_as(dp), int(order), out):
        raise RuntimeError(_err())
    return {f: np.array([getattr(out[i], f) for i in range(n)]) for f, _ in SegInfo._fields_}


def n_threads_default():
    return os.cpu_count() or 1
