"""Host-side checks of the C ABI: the library loads without a GPU, exports
every function include/dpm.h declares, the ctypes structs match the C layout
(checked by compiling a probe with gcc), and the binding fails loudly when
the library is missing (no CPU fallback exists)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1811_03557_gb300 import abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(abi.LIB_PATH):
        from paper_1811_03557_gb300 import build
        build.build()
    return abi.lib()


def test_every_declared_function_is_exported(built):
    names = abi.header_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(built, n), n
        assert n in abi._SIGS, f"binding lacks {n}"


def test_last_error_is_empty_string_initially(built):
    assert isinstance(abi.dpm_last_error(), str)


def test_invalid_arguments_are_rejected_without_gpu(built):
    with pytest.raises(abi.DPMError) as e:
        abi._check(built.dpm_ctx_create(0, None))   # NULL out-pointer: rejected before any CUDA call
    assert e.value.code == abi.DPM_EINVAL


STRUCTS = {
    "dpm_geom": (abi.dpm_geom, ["kind", "center", "axes"]),
    "dpm_gaussian": (abi.dpm_gaussian, ["amp", "alpha", "center", "zscale"]),
    "dpm_bep_info": (abi.dpm_bep_info, ["N", "lo", "h", "sigma", "ncol", "n_mplus", "n_shell"]),
    "dpm_pks_params": (abi.dpm_pks_params, ["geom", "N", "lo", "chi", "dt_max", "K", "dt_mode", "clamp"]),
    "dpm_pks_stats": (abi.dpm_pks_stats, ["t", "dt", "step", "rebuilt", "mass", "free_energy"]),
    "dpm_dd_params": (abi.dpm_dd_params, ["center", "r1", "r2", "N1", "lo1", "hi1", "N2", "lo2", "hi2",
                                          "KZ", "KG", "precision"]),
    "dpm_dd_info": (abi.dpm_dd_info, ["N", "h", "precision", "n_mplus", "n_gin", "n_gamma", "nz", "ng",
                                      "ncol", "sigma"]),
    "dpm_dd2_params": (abi.dpm_dd2_params, ["center", "R", "rz", "zoff", "N1", "lo1", "hi1", "origin1", "N2",
                                            "lo2", "hi2", "origin2", "MZ", "MG", "precision"]),
    "dpm_dd2_info": (abi.dpm_dd2_info, ["N", "h", "precision", "n_mplus", "n_gin", "n_gamma", "n_rows",
                                        "n_wedge", "ncol", "sigma"]),
    "dpm_ml_params": (abi.dpm_ml_params, ["center", "L", "radii", "N", "lo", "hi", "K", "KG", "precision"]),
    "dpm_ml_info": (abi.dpm_ml_info, ["L", "N", "h", "precision", "n_mplus", "n_gin", "n_gamma", "ncol",
                                      "sigma"]),
}


def test_struct_layout_matches_header(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dpm.h"', "int main(void){"]
    for s, (_, fields) in STRUCTS.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
                    str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for s, (cls, fields) in STRUCTS.items():
        assert int(out[s]) == ctypes.sizeof(cls), s
        for f in fields:
            assert int(out[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(abi, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(abi, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        abi.lib()
