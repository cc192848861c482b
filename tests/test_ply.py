"""PLY scene assets (Sec. 3.1): the 3DGS layout read into this library's
arrays, checked on files built byte by byte here (not by the writer)."""
import numpy as np
import pytest

from paper_2604_12626_gb300 import ply, synth


def _raw_ply(path, n, k_rest, extra_prefix=()):
    """A 3DGS-style PLY whose every property value encodes its own identity."""
    names = list(extra_prefix) + ["x", "y", "z", "f_dc_0", "f_dc_1", "f_dc_2"]
    names += [f"f_rest_{i}" for i in range(3 * k_rest)] + ["opacity", "scale_0", "scale_1", "scale_2"]
    names += ["rot_0", "rot_1", "rot_2", "rot_3"]
    vals = np.zeros((n, len(names)), np.float32)
    for j, nm in enumerate(names):
        vals[:, j] = 1000.0 * np.arange(n) + j  # row r, property j
    hdr = "ply\nformat binary_little_endian 1.0\ncomment test\nelement vertex %d\n" % n
    hdr += "".join(f"property float {nm}\n" for nm in names) + "end_header\n"
    with open(path, "wb") as f:
        f.write(hdr.encode("ascii"))
        f.write(vals.astype("<f4").tobytes())
    return names, vals


@pytest.mark.parametrize("k_rest", [15, 3, 0])
def test_read_3dgs_layout(tmp_path, k_rest):
    p = tmp_path / "a.ply"
    names, vals = _raw_ply(p, 4, k_rest, extra_prefix=("nx", "ny", "nz"))
    col = {nm: vals[:, j] for j, nm in enumerate(names)}
    g = ply.read_gaussians(str(p))
    np.testing.assert_array_equal(g["means"], np.stack([col["x"], col["y"], col["z"]], 1))
    np.testing.assert_array_equal(g["quats"][:, 0], col["rot_0"])  # w first
    np.testing.assert_array_equal(g["log_scales"][:, 2], col["scale_2"])
    np.testing.assert_array_equal(g["opacity_logits"], col["opacity"])
    for c in range(3):
        np.testing.assert_array_equal(g["sh"][:, 0, c], col[f"f_dc_{c}"])
        for i in range(15):
            want = col[f"f_rest_{c * k_rest + i}"] if i < k_rest else np.zeros(4, np.float32)
            np.testing.assert_array_equal(g["sh"][:, 1 + i, c], want)  # channel-major in the file
    assert g["sh"].shape == (4, 16, 3) and g["sh"].dtype == np.float32


def test_round_trip(tmp_path):
    g = synth.box_scene(300, seed=3)
    p = tmp_path / "b.ply"
    ply.write_gaussians(str(p), g)
    h = ply.read_gaussians(str(p))
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        np.testing.assert_array_equal(h[k], np.asarray(g[k], np.float32))


def test_rejects_ascii(tmp_path):
    p = tmp_path / "c.ply"
    p.write_bytes(b"ply\nformat ascii 1.0\nelement vertex 1\nproperty float x\nend_header\n0\n")
    with pytest.raises(ValueError, match="binary_little_endian"):
        ply.read_gaussians(str(p))
