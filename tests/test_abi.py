"""CPU checks of the C ABI: the library builds, loads, exports every function include/tgs.h
declares, and the ctypes structures have the header's layout. No CUDA call is made."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2501_14534_gb300 import build as tgs_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tgs.h")


@pytest.fixture(scope="module")
def lib():
    tgs_build.build()
    from paper_2501_14534_gb300 import _binding
    return _binding


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(tgs_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib.lib, n), n
    # and the binding declares a prototype for each
    assert set(names) <= set(lib.SIGNATURES), set(names) - set(lib.SIGNATURES)


def test_struct_layouts_match_header(lib, tmp_path):
    structs = {"tgs_config": lib.tgs_config, "tgs_gaussians": lib.tgs_gaussians,
               "tgs_camera": lib.tgs_camera, "tgs_view_out": lib.tgs_view_out,
               "tgs_grads": lib.tgs_grads, "tgs_stats": lib.tgs_stats,
               "tgs_half_params": lib.tgs_half_params, "tgs_peaks": lib.tgs_peaks}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tgs.h"', "int main(void){"]
    for s, cls in structs.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for s, cls in structs.items():
        assert int(out[s]) == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(out[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_default_config_and_status_strings(lib):
    cfg = lib.tgs_config()
    lib.lib.tgs_default_config(C.byref(cfg))
    assert (cfg.tile, cfg.ppt, cfg.support) == (16, 1, lib.TGS_SUPPORT_BOX3)
    assert abs(cfg.low_pass - 0.3) < 1e-7          # s = 0.3 (progressive-scale section)
    assert abs(cfg.eps_mask - 0.05) < 1e-7 and abs(cfg.eps_sh - 0.1) < 1e-7
    assert abs(cfg.ssim_lambda - 0.2) < 1e-7
    for s in range(8):
        assert lib.lib.tgs_status_string(s)
    assert lib.lib.tgs_status_string(99) == b"unknown status"


def test_oracle_and_product_share_no_code():
    """The oracle's C source and the CUDA sources include nothing of each other."""
    csrc = os.path.join(ROOT, "paper_2501_14534_gb300", "csrc")
    orc = open(os.path.join(ROOT, "oracle", "tgs_oracle.c")).read()
    assert "tgs.h" not in orc and "csrc" not in orc
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f
    for f in ("rasterizer.py", "_binding.py", "build.py", "synth.py"):
        txt = open(os.path.join(ROOT, "paper_2501_14534_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f


def paper_constants():
    path = os.path.join(ROOT, "tests", "golden", "paper_constants.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, value, cite = line.split(None, 2)
            assert cite.startswith("Sec. "), line
            out[name] = float(value)
    return out


def test_defaults_are_the_papers_constants(lib):
    import inspect

    import oracle
    from paper_2501_14534_gb300 import rasterizer as R
    pc = paper_constants()
    cfg = lib.tgs_config()
    lib.lib.tgs_default_config(C.byref(cfg))
    st = oracle.Settings()
    ctor = inspect.signature(R.Rasterizer.__init__).parameters
    for name, lib_v, orc_v in [("eps_mask", cfg.eps_mask, st.eps_mask), ("eps_sh", cfg.eps_sh, st.eps_sh),
                               ("low_pass", cfg.low_pass, st.low_pass)]:
        assert abs(lib_v - pc[name]) < 1e-7 and orc_v == pc[name] and ctor[name].default == pc[name], name
    q = pc["significance_quantile"]
    assert inspect.signature(R.Rasterizer.significance).parameters["quantile"].default == q
    assert inspect.signature(oracle.significance).parameters["quantile"].default == q
    fr = R.Rasterizer.pruning_fractions()
    assert len(fr) == pc["prune_rounds"] and fr[0] == pc["first_prune_fraction"]
    assert all(abs(b / a - pc["prune_decay"]) < 1e-12 for a, b in zip(fr, fr[1:]))
    assert oracle.SSIM_WINDOW == pc["ssim_window"]
    for name, lib_v, orc_v in [("lambda_mask", cfg.lambda_mask, oracle.MASK_LAMBDA),
                               ("lambda_sh_mask", cfg.lambda_sh_mask, oracle.SH_MASK_LAMBDA)]:
        assert abs(lib_v - pc[name]) < 1e-7 and orc_v == pc[name] and ctor[name].default == pc[name], name
