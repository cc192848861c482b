"""Host-side checks of the C ABI (no GPU): the library builds and loads,
exports every function include/gs.h declares, the ctypes mirrors have the C
layouts, and argument errors are caught on the host."""
import ctypes
import re
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "gs.h"


@pytest.fixture(scope="module")
def lib():
    from paper_2604_12626_gb300 import build

    return build.build()


def declared_functions():
    txt = HEADER.read_text()
    return sorted(set(re.findall(r"^(?:gs_status|int32_t)\s+(gs_\w+)\s*\(", txt, re.M)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", str(lib)], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(gs_\w+)$", out, re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(str(lib))
    for n in names:
        assert hasattr(L, n)
    from paper_2604_12626_gb300 import api

    assert set(api.EXPORTS) == set(names)


def test_ctypes_structs_match_c_layout(tmp_path, lib):
    from paper_2604_12626_gb300 import api

    structs = {"gs_camera": api.GsCamera, "gs_gaussians": api.GsGaussians, "gs_batch": api.GsBatch,
               "gs_render_config": api.GsRenderConfig, "gs_stats": api.GsStats, "gs_avatars": api.GsAvatars,
               "gs_ws_sections": api.GsWsSections, "gs_mesh": api.GsMesh}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _t in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _t in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_host_side_argument_checks(lib):
    from paper_2604_12626_gb300 import api, synth

    b = api.Batch(np.array([0, 10, 30]))
    assert api.workspace_size(api.make_config(64, 48), b) > 0
    for bad in [dict(tile=(7, 7)), dict(batch_depth=1000), dict(tile=(64, 32))]:
        with pytest.raises(api.GsError, match="INVALID_ARG"):
            api.workspace_size(api.make_config(64, 48, **bad), b)
    with pytest.raises(api.GsError, match="INVALID_ARG"):
        api.workspace_size(api.make_config(0, 48), b)
    with pytest.raises(api.GsError, match="INVALID_ARG"):
        api.workspace_size(api.make_config(64, 48), api.Batch(np.array([0, 10, 5])))
    with pytest.raises(api.GsError, match="INVALID_ARG"):
        api.workspace_size(api.make_config(64, 48), api.Batch(np.array([0, 10]), view_env=[3]))
    # the full 64-env batch fits a GB300 comfortably
    sizes = synth.batch_sizes(64)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    assert api.workspace_size(api.make_config(256, 256), api.Batch(offs)) < 40e9


def test_no_cpu_fallback(lib):
    torch = pytest.importorskip("torch")
    from paper_2604_12626_gb300 import api

    cpu = torch.zeros((4, 3))
    with pytest.raises(ValueError, match="CUDA"):
        api.Gaussians(cpu, cpu, torch.zeros((4, 4)), torch.zeros(4), torch.zeros((4, 16, 3)))
