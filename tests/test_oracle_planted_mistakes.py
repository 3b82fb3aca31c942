"""Planted mistakes in the FP64 oracle must fail its pins.

Each case copies ``oracle/fs4d_oracle.cpp``, plants one plausible mistake (a
dropped term, a flipped sign, a transposed operand or index, a shifted offset, a
threshold taken on the wrong side), builds the copy into a temporary library
and runs the oracle's pin tests (``test_oracle_pins.py``,
``test_oracle_backward.py``, ``test_oracle_densify.py``) against it.  A mistake that every pin lets through
shows a pin that is missing.  The real oracle is never modified.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fs4d_oracle.cpp")
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_backward.py", "tests/test_oracle_densify.py"]

# (name, text in the oracle, replacement, which occurrence of the text).  Texts that
# the forward and the backward share are planted in their first occurrence, the
# forward one (the file defines the forward first).
MISTAKES = [
    # Eq. 5: HexPlane sampling and fusion
    ("plane axis pairs xz and yz swapped", "{{0, 1}, {0, 2}, {1, 2}, {0, 3}",
     "{{0, 1}, {1, 2}, {0, 2}, {0, 3}", 0),
    ("time not mapped to [-1, 1]", "c[3] = 2.0 * t - 1.0;", "c[3] = t;", 0),
    ("box normalised to [0, 1]", "c[a] = 2.0 * (xyz[a] - s->aabb_min[a]) / (s->aabb_max[a] - s->aabb_min[a]) - 1.0;",
     "c[a] = (xyz[a] - s->aabb_min[a]) / (s->aabb_max[a] - s->aabb_min[a]);", 0),
    ("grid vertices at cell centres", "double g = (uc + 1.0) * 0.5 * (R - 1);",
     "double g = (uc + 1.0) * 0.5 * R - 0.5;", 0),
    ("bilinear corner transposed", "v10 = P[((int64_t)j0 * Ra + i0 + 1) * h + c]",
     "v10 = P[((int64_t)(j0 + 1) * Ra + i0) * h + c]", 0),
    ("bilinear weights transposed", "fa * (1 - fb) * v10 + (1 - fa) * fb * v01",
     "(1 - fa) * fb * v10 + fa * (1 - fb) * v01", 0),
    ("border clamping dropped", "double uc = std::min(1.0, std::max(-1.0, u));", "double uc = u;", 0),
    ("planes summed instead of multiplied", "for (int k = 0; k < h; ++k) f[k] *= v[k];",
     "for (int k = 0; k < h; ++k) f[k] += v[k];", 0),
    # Sec. 4.2: MLP and heads; Eq. 6
    ("bias dropped", "double acc = s->mlp[L.b[k] + o];", "double acc = 0.0;", 0),
    ("weight matrix transposed", "s->mlp[L.w[k] + (int64_t)o * L.in[k] + i]",
     "s->mlp[L.w[k] + (int64_t)i * L.out[k] + o]", 0),
    ("ReLU after the first layer dropped", "for (auto& v : a1) v = relu(v);", "", 0),
    ("scale head reads the rotation columns", "delta[10 * g + 7 + a]", "delta[10 * g + 6 + a]", 0),
    # Eq. 2 / Eq. 3 and the colour
    ("rotation entry with the wrong sign", "R[0][1] = 2 * (x * y - w * z);", "R[0][1] = 2 * (x * y + w * z);", 0),
    ("covariance R^T S^2 R", "acc += R[i][k] * S[k] * S[k] * R[j][k];", "acc += R[k][i] * S[k] * S[k] * R[k][j];", 0),
    ("quaternion not normalised", "for (int k = 0; k < 4; ++k) q[k] /= qn;", "", 0),
    ("Jacobian third column sign", "-cam->fx * txz / (p[2] * p[2])", "cam->fx * txz / (p[2] * p[2])", 0),
    ("low-pass dilation dropped", "double a = C2[0][0] + kDilation, b = C2[0][1], c = C2[1][1] + kDilation;",
     "double a = C2[0][0], b = C2[0][1], c = C2[1][1];", 0),
    ("conic off-diagonal sign", "out->conic[3 * (int64_t)g + 1] = -b / det;",
     "out->conic[3 * (int64_t)g + 1] = b / det;", 0),
    ("radius from the smaller eigenvalue", "double lmax = mid + std::sqrt", "double lmax = mid - std::sqrt", 0),
    ("2-sigma radius", "double r3 = 3.0 * std::sqrt(lmax);", "double r3 = 2.0 * std::sqrt(lmax);", 0),
    ("tile rectangle end not exclusive", "x1 = (int)std::floor((u + radius) / tile) + 1;",
     "x1 = (int)std::floor((u + radius) / tile);", 0),
    ("no guard band on the Jacobian", "const double kGuard = 1.3;", "const double kGuard = 1e9;", 0),
    ("view direction reversed", "dir[k] = X[k] - campos[k];", "dir[k] = campos[k] - X[k];", 0),
    ("view direction from the canonical mean", "dir[k] = X[k] - campos[k];",
     "dir[k] = (double)s->means[3 * (int64_t)g + k] - campos[k];", 0),
    ("frame deformed at a fixed time", "orc_deform(s, t, X.data(), Q.data(), Sc.data());",
     "orc_deform(s, 0.5, X.data(), Q.data(), Sc.data());", 0),
    ("opacity sigmoid sign", "out->opacity[g] = 1.0 / (1.0 + std::exp(-logit));",
     "out->opacity[g] = 1.0 / (1.0 + std::exp(logit));", 0),
    ("camera centre sign", "campos[c] = -(Rc[0][c] * tc[0]", "campos[c] = (Rc[0][c] * tc[0]", 0),
    ("colour offset 0.5 dropped", "double acc = 0.5;", "double acc = 0.0;", 0),
    ("SH with the Condon-Shortley phase", "Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;",
     "Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;", 0),
    ("SH degree-2 term sign", "0.25 * std::sqrt(15.0 / PI) * (x * x - y * y)",
     "0.25 * std::sqrt(15.0 / PI) * (y * y - x * x)", 0),
    ("SH degree-3 coefficient", "Y[12] = 0.25 * std::sqrt(7.0 / PI) * z * (5.0 * z * z - 3.0);",
     "Y[12] = 0.25 * std::sqrt(7.0 / PI) * z * (5.0 * z * z - 1.0);", 0),
    # Tile keys, sort, ranges
    ("sort descending", "return a.first < b.first;", "return a.first > b.first;", 0),
    ("tile field shifted", "pairs.push_back({(tile_id << 32) | depth_bits[g], (uint32_t)g});",
     "pairs.push_back({(tile_id << 31) | depth_bits[g], (uint32_t)g});", 0),
    ("range end inclusive", "ranges[2 * tile_id + 1] = (uint32_t)(i + 1);",
     "ranges[2 * tile_id + 1] = (uint32_t)i;", 0),
    # Eq. 1 / Eq. 4 compositing (the tiled blend; the brute-force restatement keeps the right rule)
    ("pixel corner instead of centre", "int last = 0;\n    const double cx = px + 0.5, cy = py + 0.5;",
     "int last = 0;\n    const double cx = px, cy = py;", 0),
    ("Gaussian cross term sign", "- conic[3 * g + 1] * dx * dy;", "+ conic[3 * g + 1] * dx * dy;", 0),
    ("alpha not clamped at 0.99", "const double alpha = std::min(kAlphaMax, a_raw);",
     "const double alpha = a_raw;", 0),
    ("1/255 skip dropped", "if (alpha < kAlphaMin) continue;", "", 0),
    ("stop after the crossing term", "if (Tn < kTMin) break;", "if (T < kTMin) break;", 0),
    ("colour weighted by the transmittance behind", "C[ch] += rgb[3 * g + ch] * alpha * T;",
     "C[ch] += rgb[3 * g + ch] * alpha * Tn;", 0),
    # The backward's chain rule (caught by the central differences)
    ("backward: mean gradient cross term sign", "g_xy[2 * g] += dpow * (-(A * dx + B * dy));",
     "g_xy[2 * g] += dpow * (-(A * dx - B * dy));", 0),
    ("backward: terms behind dropped from dL/dalpha",
     "dL_dalpha += dC[ch] * (rgb[3 * g + ch] * Ti - behind[ch] / (1.0 - alpha));",
     "dL_dalpha += dC[ch] * (rgb[3 * g + ch] * Ti);", 0),
    ("backward: transmittance not restored", "const double Ti = T / (1.0 - alpha);", "const double Ti = T;", 0),
    ("backward: inverse gradient sign", "GS2[i][j] = -acc;", "GS2[i][j] = acc;", 0),
    ("backward: Jacobian derivative factor", "gp[2] += gJ[0][2] * (2.0 * cam->fx * p[0] / (pz2 * pz));",
     "gp[2] += gJ[0][2] * (cam->fx * p[0] / (pz2 * pz));", 0),
    ("backward: rotation derivative sign", "{2 * y, -4 * x, -2 * w}", "{2 * y, -4 * x, 2 * w}", 0),
    ("backward: quaternion normalisation ignored", "gQ[4 * (int64_t)g + c] += (gqh[c] - qh[c] * qd) / qn;",
     "gQ[4 * (int64_t)g + c] += gqh[c] / qn;", 0),
    ("backward: exp of the log-scale dropped", "gS[3 * (int64_t)g + k] += gsc[k] * sc[k];",
     "gS[3 * (int64_t)g + k] += gsc[k];", 0),
    ("backward: sigmoid derivative dropped", "G->opacity_logits[g] += g_op[g] * op[g] * (1.0 - op[g]);",
     "G->opacity_logits[g] += g_op[g] * op[g];", 0),
    ("backward: SH basis derivative", "dY[12][2] = h * (15.0 * z * z - 3.0);", "dY[12][2] = h * (5.0 * z * z - 3.0);", 0),
    ("backward: ReLU mask of phi_d dropped", "const double gpre = FD[o] > 0.0 ? gfd[o] : 0.0;",
     "const double gpre = gfd[o];", 0),
    ("backward: plane gradient weights transposed", "G->planes[off + e10] += gv * fa[p] * (1 - fb[p]);",
     "G->planes[off + e10] += gv * (1 - fa[p]) * fb[p];", 0),
    ("backward: box scale of the sampling point", "G->means[3 * (int64_t)g + a] += gv * dv_dfa * da[p] * 2.0 /",
     "G->means[3 * (int64_t)g + a] += gv * dv_dfa * da[p] * 1.0 /", 0),
    ("backward: projected-mean gradient sign", "G->xy[i] += g_xy[i];", "G->xy[i] -= g_xy[i];", 0),
    # App. B: colour and opacity heads
    ("colour head replaces the SH instead of adding", "for (int j = 0; j < K3; ++j) sh[(int64_t)g * K3 + j] += dc[j];",
     "for (int j = 0; j < K3; ++j) sh[(int64_t)g * K3 + j] = dc[j];", 0),
    ("opacity head reads the colour head's hidden layer", "    linear(s, Lo, 10, fd.data(), hid.data());\n", "", 0),
    ("colour head without its ReLU", "for (auto& v : hid) v = relu(v);", "", 1),
    ("projection ignores the deformed colour", "acc += Y[k] * (shd ? shd[e] : (double)s->sh[e]);",
     "acc += Y[k] * (double)s->sh[e];", 0),
    # App. A: densification and pruning
    ("densify: children keep the parent's scale", "for (int k = 0; k < 3; ++k) log_scales[3 * o + k] -= shrink;",
     "", 0),
    ("densify: copies not made", "if (cls[i] == 2) out.push_back({i, 1});", "if (cls[i] == 5) out.push_back({i, 1});",
     0),
    ("densify: threshold taken strictly", "const bool selected = avg >= grad_threshold;",
     "const bool selected = avg > grad_threshold;", 0),
    ("densify: child offset rotated by R^T",
     "means[3 * o + r] += R[r][0] * sz[0] + R[r][1] * sz[1] + R[r][2] * sz[2];",
     "means[3 * o + r] += R[0][r] * sz[0] + R[1][r] * sz[1] + R[2][r] * sz[2];", 0),
    ("densify: log-scale used as the scale", "sz[k] = std::exp((double)s->log_scales[3 * i + k]) * (double)z[k];",
     "sz[k] = (double)s->log_scales[3 * i + k] * (double)z[k];", 0),
    ("densify: split Gaussian also kept", "if (cls[i] == 1 || cls[i] == 2) out.push_back({i, 0});",
     "if (cls[i] >= 1) out.push_back({i, 0});", 0),
    ("densify: transparent Gaussians still densified", "if (s->opacity_logits[i] < prune_logit) cls[i] = 0;",
     "if (s->opacity_logits[i] < prune_logit && !selected) cls[i] = 0;", 0),
    ("densify: both children from one draw", "const float* z = normals + 6 * i + 3 * (kd - 2);",
     "const float* z = normals + 6 * i;", 0),
]


def _plant(text: str, old: str, new: str, nth: int) -> str:
    pos = -1
    for _ in range(nth + 1):
        pos = text.find(old, pos + 1)
        assert pos >= 0, f"the oracle no longer contains {old!r}"
    return text[:pos] + new + text[pos + len(old):]


def _run(idx: int, workdir: str) -> tuple:
    name, old, new, nth = MISTAKES[idx]
    src = os.path.join(workdir, f"m{idx}.cpp")
    lib = os.path.join(workdir, f"m{idx}.so")
    with open(SRC) as f:
        text = f.read()
    with open(src, "w") as f:
        f.write(_plant(text, old, new, nth))
    subprocess.run(["g++", "-O1", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-I", os.path.dirname(SRC),
                    "-o", lib, src], check=True, capture_output=True)
    env = dict(os.environ, FS4D_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PIN_FILES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
    return r.returncode, failed, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    work = str(tmp_path_factory.mktemp("planted"))
    workers = max(2, min(16, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        futs = {i: ex.submit(_run, i, work) for i in range(len(MISTAKES))}
        return {i: f.result() for i, f in futs.items()}


def test_every_planted_text_is_present():
    with open(SRC) as f:
        text = f.read()
    for name, old, new, nth in MISTAKES:
        assert text.count(old) >= nth + 1, name


@pytest.mark.parametrize("idx", range(len(MISTAKES)), ids=[m[0] for m in MISTAKES])
def test_planted_mistake_fails_a_pin(outcomes, idx):
    rc, failed, tail = outcomes[idx]
    # exit status 1: the pins ran and at least one failed (not a crash or a collection error)
    assert rc == 1 and failed, f"{MISTAKES[idx][0]}: no pin failed (exit {rc})\n{tail}"
