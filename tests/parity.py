"""Frame parity against the FP64 oracle, pixel by pixel (test helper).

Every pixel of a GPU frame must equal the oracle's frame within `tol`, or else
equal, within `tol`, one of the other results the oracle enumerates for that
pixel: the blends in which the pixel's decisions that lie within float32
rounding of their thresholds are taken the other way (alpha vs 1/255 and T vs
1e-4 within `rel_tol` relative, two blended depths within `depth_tol`), over
the tile lists in which the Gaussians whose tile-rectangle decision lies within
`px_tol` pixels of its integer boundary are in or out of the pixel's tile.
Nothing is excluded: a pixel that matches none of these fails.
"""
import numpy as np

import oracle


def oracle_frame(scene, cam, t, deform=True, tile=16):
    """The oracle's frame and the pieces its per-pixel outcomes need."""
    img, T, nc, mg, K = oracle.render(scene, cam, t, deform=deform, tile=tile)
    if deform:
        X, Q, S = oracle.deform(scene, t)
        if getattr(scene, "color_heads", False):  # App. B: deformed colour and opacity
            shd, lgd = oracle.appearance(scene, t)
            p = oracle.project(scene, cam, X, Q, S, tile=tile, sh=shd, opacity_logits=lgd)
        else:
            p = oracle.project(scene, cam, X, Q, S, tile=tile)
    else:
        p = oracle.project(scene, cam, tile=tile)
    tx, ty = (cam.width + tile - 1) // tile, (cam.height + tile - 1) // tile
    dbits = oracle.depth_bits(p["depth"])
    _, vals, ranges = oracle.bin_sort(dbits, p["rect"], tx, ty)
    return dict(img=img, T=T, nc=nc, margin=mg, K=K, proj=p, values=vals, ranges=ranges, dbits=dbits, tx=tx,
                tile=tile)


def _toggled(base, gs, mask, dbits):
    """base with the Gaussians gs[b] (bit b of mask) added or removed, in (depth, index) order."""
    s = set(int(g) for g in base)
    for b, g in enumerate(gs):
        if mask & (1 << b):
            s ^= {int(g)}
    return np.array(sorted(s, key=lambda g: (int(dbits[g]), g)), np.uint32)


def pixel_matches(value, px, py, base, gs, proj, dbits, tol, rel_tol, depth_tol, T=None, nc=None):
    """Whether `value` (with T, nc if given) equals, within tol, one of the oracle's
    outcomes for pixel (px, py) over its tile list `base`, with the Gaussians gs
    (uncertain members of the tile) in or out of the list."""
    for mask in range(1 << len(gs)):
        lst = base if mask == 0 else _toggled(base, gs, mask, dbits)
        outs = oracle.pixel_outcomes(lst, px, py, proj, rel_tol, depth_tol)
        if outs is None:  # many near-threshold decisions (long lists): enumerate more of them
            outs = oracle.pixel_outcomes(lst, px, py, proj, rel_tol, depth_tol, max_flip=12)
        if outs is None:
            continue
        good = np.abs(outs[:, :3] - value).max(1) <= tol
        if T is not None:
            good &= np.abs(outs[:, 3] - T) <= tol
        if nc is not None:
            good &= (outs[:, 4] == nc) | np.array([_position_tie(lst, int(o), int(nc), proj, depth_tol)
                                                   for o in outs[:, 4]])
        if good.any():
            return True
    return False


def _position_tie(lst, last, nc, proj, depth_tol):
    """The last contributor's list position depends on the order of equal-depth
    terms, including ones that do not blend at this pixel: position `last` (1-based)
    may read as `nc` when the terms between them tie in depth with it."""
    if last == nc or last < 1 or nc < 1 or abs(nc - last) > 2:
        return False
    d = proj["depth"][np.asarray(lst, np.int64)]
    lo, hi = min(last, nc) - 1, max(last, nc) - 1
    ref = d[last - 1]
    return bool(np.all(np.abs(d[lo:hi + 1] - ref) <= depth_tol * abs(ref)))


def tile_list(proj, dbits, tiles_x, t_id):
    """The oracle's list of tile t_id: the Gaussians whose rectangle holds it, in
    (float32 depth, index) order."""
    r = proj["rect"]
    tx, ty = t_id % tiles_x, t_id // tiles_x
    g = np.flatnonzero((r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3]))
    return g[np.lexsort((g, dbits[g]))].astype(np.uint32)


def check_frame(img, fr, T=None, nc=None, tol=1e-4, rel_tol=5e-5, px_tol=2e-4, depth_tol=1e-6,
                max_members=4):
    """Checks every pixel of img ([H][W][3]; T, nc optional) against the oracle
    frame fr; returns statistics.  `unresolved` pixels match no outcome."""
    H, W = img.shape[:2]
    tile, tx = fr["tile"], fr["tx"]
    p, vals, ranges, dbits = fr["proj"], fr["values"], fr["ranges"], fr["dbits"]
    err = np.abs(img - fr["img"]).max(2)
    off = err > tol
    if T is not None:
        off |= np.abs(T - fr["T"]) > tol
    if nc is not None:
        off |= nc != fr["nc"]
    members = oracle.uncertain_memberships(p, W, H, px_tol, tile)
    resolved = unresolved = 0
    worst = 0.0
    for py, px in zip(*np.nonzero(off)):
        t_id = (py // tile) * tx + px // tile
        base = vals[ranges[t_id, 0]:ranges[t_id, 1]]
        gs = members.get(int(t_id), [])[:max_members]
        ok = pixel_matches(img[py, px], px, py, base, gs, p, dbits, tol, rel_tol, depth_tol,
                           None if T is None else T[py, px], None if nc is None else nc[py, px])
        if ok:
            resolved += 1
        else:
            unresolved += 1
            worst = max(worst, float(err[py, px]))
    n = H * W
    stats = {"pixels": n, "max_err_on_base": float(err[~off].max()) if (~off).any() else 0.0,
             "other_outcome": int(resolved), "other_outcome_frac": resolved / n,
             "unresolved": int(unresolved), "worst_unresolved": worst,
             "near_threshold_pixels": int((fr["margin"] < rel_tol).sum()),
             "uncertain_member_tiles": len(members)}
    print("frame parity:", stats)
    return stats


def oracle_frame_composed(scenes, shifts, cam, t, tile=16):
    """The oracle's frame of several scenes composed (Sec. 5.4), as oracle_frame."""
    p = oracle.project_composed(scenes, shifts, cam, t, tile=tile)
    img, T, nc, mg, vals, ranges = oracle.composite_projected(p, cam, tile=tile)
    tx = (cam.width + tile - 1) // tile
    return dict(img=img, T=T, nc=nc, margin=mg, K=len(vals), proj=p, values=vals, ranges=ranges,
                dbits=oracle.depth_bits(p["depth"]), tx=tx, tile=tile)
