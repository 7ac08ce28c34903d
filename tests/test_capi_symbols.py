"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/heart.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "heart.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:heart_status|const char \*)\s*(heart_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("heart_spectrometer_create", "heart_trace", "heart_submit", "heart_poll", "heart_last_error"):
        assert n in names


def test_library_builds_loads_and_exports_all_symbols():
    from paper_2503_16955_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    import paper_2503_16955_gb300 as H
    assert sorted(H.EXPORTS) == declared_functions()


def _c_layout(tmp_path):
    """sizeof / offsetof of the public structs as the C compiler lays them out"""
    import subprocess
    structs = {
        "heart_tally": ["refl_hist", "collisions"],
        "heart_spectral_component": ["weight"],
        "heart_source_desc": ["spot_fwhm_mm", "polarization", "table_keV", "n_table"],
        "heart_ray_arrays": ["energy_keV", "pol_z"],
        "heart_qe_table": ["n"],
        "heart_spectrometer_desc": ["pixel_mm", "count_type", "sampler", "thin_vstar", "n_orders",
                                    "order_K_rel", "irc_e_keV", "irc_e_shift_rad"],
        "heart_tune": ["rays_per_s"],
        "heart_ray_record": ["u_mm", "no_bragg", "pol"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "heart.h"', "int main(void) {"]
    for st, fields in structs.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (l.split() for l in out.splitlines())}, structs


def test_binding_structs_match_header_layout(tmp_path):
    import paper_2503_16955_gb300 as H
    lay, structs = _c_layout(tmp_path)
    for st, fields in structs.items():
        if st == "heart_ray_record":
            assert H.RECORD_DTYPE.itemsize == lay[st]
            for f in fields:
                assert H.RECORD_DTYPE.fields[f][1] == lay[f"{st}.{f}"], f
            continue
        cls = getattr(H, st)
        assert ctypes.sizeof(cls) == lay[st], st
        for f in fields:
            assert getattr(cls, f).offset == lay[f"{st}.{f}"], (st, f)


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2503_16955_gb300 as H
    with pytest.raises(RuntimeError):
        H.library(str(tmp_path / "missing.so"))
