"""Reading and writing 3DGS scene assets in PLY format (Sec. 3.1: the scene
pipeline prepares 3DGS assets as standard PLY files).

The layout is the one 3DGS tools write: a binary little-endian PLY with one
`vertex` element per Gaussian and float32 properties
    x y z  [nx ny nz]  f_dc_0..2  f_rest_0..(3 K - 1)  opacity
    scale_0..2  rot_0..3
where f_dc are the degree-0 SH coefficients (R, G, B), f_rest the higher
bands stored channel-major (all K coefficients of R, then of G, then of B),
opacity the logit, scale the log-scales and rot the quaternion (w, x, y, z).
Here the arrays are returned as this library takes them: sh [N, 16, 3] with
the channel fastest (coefficient l^2 + l + m, channel c at [.., i, c]).  Host
code only (NumPy); nothing here runs on the render path.
"""
from __future__ import annotations

import numpy as np

_TYPES = {"float": "<f4", "float32": "<f4", "double": "<f8", "float64": "<f8", "uchar": "u1", "uint8": "u1",
          "char": "i1", "int8": "i1", "ushort": "<u2", "uint16": "<u2", "short": "<i2", "int16": "<i2",
          "uint": "<u4", "uint32": "<u4", "int": "<i4", "int32": "<i4"}


def read_gaussians(path: str, sh_degree: int = 3) -> dict:
    """Gaussians of a 3DGS PLY file: means [N,3], log_scales [N,3], quats
    [N,4] (w, x, y, z), opacity_logits [N], sh [N,16,3] (float32; bands above
    the file's degree are zero)."""
    with open(path, "rb") as f:
        if f.readline().strip() != b"ply":
            raise ValueError(f"{path}: not a PLY file")
        fmt, n, props, in_vertex = None, None, [], False
        while True:
            line = f.readline()
            if not line:
                raise ValueError(f"{path}: header without end_header")
            tok = line.decode("ascii").split()
            if not tok:
                continue
            if tok[0] == "format":
                fmt = tok[1]
            elif tok[0] == "element":
                in_vertex = tok[1] == "vertex"
                if in_vertex:
                    n = int(tok[2])
                elif n is None:
                    raise ValueError(f"{path}: elements before 'vertex' are not supported")
            elif tok[0] == "property" and in_vertex:
                if tok[1] == "list":
                    raise ValueError(f"{path}: list properties in 'vertex' are not supported")
                props.append((tok[2], _TYPES[tok[1]]))
            elif tok[0] == "end_header":
                break
        if fmt != "binary_little_endian":
            raise ValueError(f"{path}: only binary_little_endian PLY is supported (got {fmt})")
        if n is None:
            raise ValueError(f"{path}: no vertex element")
        data = np.fromfile(f, dtype=np.dtype(props), count=n)
    names = set(data.dtype.names)

    def col(name):
        return data[name].astype(np.float32)

    def stack(prefix, k):
        return np.stack([col(f"{prefix}{i}") for i in range(k)], axis=1)

    out = {"means": np.stack([col("x"), col("y"), col("z")], axis=1),
           "log_scales": stack("scale_", 3), "quats": stack("rot_", 4), "opacity_logits": col("opacity")}
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, 0, :] = stack("f_dc_", 3)
    n_rest = sum(1 for nm in names if nm.startswith("f_rest_"))
    if n_rest % 3:
        raise ValueError(f"{path}: {n_rest} f_rest properties is not a multiple of 3")
    k = n_rest // 3  # coefficients per channel beyond degree 0
    k_use = min(k, (sh_degree + 1) ** 2 - 1)
    if k:
        rest = stack("f_rest_", n_rest).reshape(n, 3, k)  # channel-major in the file
        sh[:, 1:1 + k_use, :] = np.transpose(rest[:, :, :k_use], (0, 2, 1))
    for key in out:
        out[key] = np.ascontiguousarray(out[key])
    out["sh"] = sh
    return out


def write_gaussians(path: str, g: dict, sh_degree: int = 3) -> None:
    """Writes Gaussians in the 3DGS PLY layout (the inverse of read_gaussians)."""
    n = int(np.asarray(g["means"]).shape[0])
    k = (sh_degree + 1) ** 2 - 1
    names = ["x", "y", "z", "nx", "ny", "nz", "f_dc_0", "f_dc_1", "f_dc_2"] + [f"f_rest_{i}" for i in range(3 * k)]
    names += ["opacity", "scale_0", "scale_1", "scale_2", "rot_0", "rot_1", "rot_2", "rot_3"]
    rec = np.zeros(n, dtype=[(nm, "<f4") for nm in names])
    m = np.asarray(g["means"], np.float32)
    rec["x"], rec["y"], rec["z"] = m[:, 0], m[:, 1], m[:, 2]
    sh = np.asarray(g["sh"], np.float32).reshape(n, 16, 3)
    for c in range(3):
        rec[f"f_dc_{c}"] = sh[:, 0, c]
        for i in range(k):
            rec[f"f_rest_{c * k + i}"] = sh[:, 1 + i, c]
    rec["opacity"] = np.asarray(g["opacity_logits"], np.float32)
    for i in range(3):
        rec[f"scale_{i}"] = np.asarray(g["log_scales"], np.float32)[:, i]
    for i in range(4):
        rec[f"rot_{i}"] = np.asarray(g["quats"], np.float32)[:, i]
    header = "ply\nformat binary_little_endian 1.0\nelement vertex %d\n" % n
    header += "".join(f"property float {nm}\n" for nm in names) + "end_header\n"
    with open(path, "wb") as f:
        f.write(header.encode("ascii"))
        rec.tofile(f)
