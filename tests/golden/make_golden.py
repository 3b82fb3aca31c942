"""Write the oracle's regression fixtures under tests/golden/.

Every stored value comes from the FP64 oracle (``oracle/``) on seeded synthetic
scenes; nothing here comes from the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py

The fixtures freeze the oracle's results for two small frames so that a change
to its arithmetic shows up as a failing test (``tests/test_golden.py``); such a
change must name, in its commit message, the passage of the paper (or the
reading of it) that justifies it.
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2310_08528_gb300 import scenegen as sg  # noqa: E402


def cases():
    """(name, scene, camera, t, description) of every fixture."""
    cam_obj = sg.hemisphere_cameras(5, width=160, height=120, seed=0)[3]
    return [
        ("tiny_seed0", sg.make_tiny(0), sg.tiny_camera(), 0.5,
         "N=2000 tiny scene (means U[-1,1]^3, log-scales N(-4,0.5), SH degree 0, HexPlane 32x32 spatial x 8 "
         "temporal x 16 features, MLP weights N(0,0.02)), 128x128 camera at (0,-4,0), t=0.5"),
        ("object_sh3_seed1", sg.make_object(1, n=3000, res_spatial=(16, 32), res_time=9, h=8, mlp_std=0.1),
         cam_obj, 0.73,
         "N=3000 object-shaped scene (32-component mixture, SH degree 3), HexPlane {16,32} x 9 x 8 features, "
         "MLP weights N(0,0.1), 160x120 hemisphere camera 3 of 5, t=0.73"),
    ]


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).astype(np.asarray(a).dtype.newbyteorder("<")).tobytes()).hexdigest()


def record(scene, cam, t):
    X, Q, S = oracle.deform(scene, t)
    p = oracle.project(scene, cam, X, Q, S)
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    keys, vals, ranges = oracle.bin_sort(oracle.depth_bits(p["depth"]), p["rect"], tx, ty)
    img, T, nc, _, K = oracle.render(scene, cam, t)
    rng = np.random.default_rng(123)
    ys = rng.integers(0, cam.height, 24)
    xs = rng.integers(0, cam.width, 24)
    lit = np.argwhere(nc > 0)
    extra = lit[rng.choice(len(lit), size=min(8, len(lit)), replace=False)]
    pix = [(int(y), int(x)) for y, x in zip(ys, xs)] + [(int(y), int(x)) for y, x in extra]
    return {
        "pairs": int(K),
        "keys_sha256": digest(keys.astype(np.uint64)),
        "values_sha256": digest(vals.astype(np.uint32)),
        "ranges_sha256": digest(ranges.astype(np.uint32)),
        "visible": int((p["radius"] > 0).sum()),
        "image_channel_sums": [float(v) for v in img.reshape(-1, 3).sum(0)],
        "pixels": [[y, x, *[float(v) for v in img[y, x]], float(T[y, x]), int(nc[y, x])] for y, x in pix],
        "deformed_first8": {"means": X[:8].tolist(), "quats": Q[:8].tolist(), "log_scales": S[:8].tolist()},
    }


def _dump(obj) -> str:
    """JSON with one line per top-level key and per pixel row (diff-friendly)."""
    lines = []
    for k, v in obj.items():
        if k == "pixels":
            rows = ",\n  ".join(json.dumps(r) for r in v)
            lines.append(f' "{k}": [\n  {rows}\n ]')
        elif k == "deformed_first8":
            inner = ",\n  ".join(f'"{a}": {json.dumps(b)}' for a, b in v.items())
            lines.append(f' "{k}": {{\n  {inner}\n }}')
        else:
            lines.append(f' "{k}": {json.dumps(v)}')
    return "{\n" + ",\n".join(lines) + "\n}\n"


def main():
    for name, scene, cam, t, desc in cases():
        out = {
            "what": "FP64 oracle results (regression fixture, written by tests/golden/make_golden.py)",
            "scene": desc,
            "computes": "Eq. 5 features, Sec. 4.2 MLP heads, Eq. 6 deformation, Eq. 2-3 projection, tile binning "
                        "and (tile, depth, index) sort, Eq. 4 / Eq. 1 compositing",
            **record(scene, cam, t),
        }
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            f.write(_dump(out))
        print(name, out["pairs"], out["visible"])


if __name__ == "__main__":
    main()
