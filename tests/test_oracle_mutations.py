"""The oracle's pins catch plausible mistakes.  Each mutant below is the
oracle's C source with one planted mistake (a sign, an index, a constant, a
dropped term or clamp, a transposed operand), one per step of the method:
Eq. 3/4 (encode, decode), the threshold test, the regularisation, Algorithms
2 and 5, the L_c reading (reconstruction, HLL, bed source, ghosts), friction,
inflow, CFL, the decode-back and the matched faces.  Every mutant must build
and must fail at least one pin of tests/test_oracle_{mra,tree,fv1,match}.py.
The mutants are built and run on the CPU, in the oracle's git-ignored build
folder (no GPU).  The CNN oracle of the learned look-ahead gets the same
treatment against its own pins, in this process."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hwfv1_oracle.c")
WORK = os.path.join(ROOT, "oracle", "_build", "mutants")
PINS = ["tests/test_oracle_mra.py", "tests/test_oracle_tree.py", "tests/test_oracle_fv1.py",
        "tests/test_oracle_match.py", "tests/test_oracle_skip.py"]

# (name, text in the oracle, the same text with the mistake)
MUTANTS = [
    ("encode_scale", "out[0] = 0.25 * (a + b);", "out[0] = 0.5 * (a + b);"),
    ("encode_detail_sign", "out[1] = 0.25 * (d + e);", "out[1] = 0.25 * (d - e);"),
    ("encode_pairing", "double a = c[0] + c[2];", "double a = c[0] + c[1];"),
    ("encode_child_index", "c[1] = ch[rm(n + 1, 2 * i + 1, 2 * j)];", "c[1] = ch[rm(n + 1, 2 * i, 2 * j + 1)];"),
    ("decode_sign", "c[2] = (s - da) + (db - dg);", "c[2] = (s - da) + (db + dg);"),
    ("threshold_level_power", "double thr = ldexp(eps, n - L);", "double thr = ldexp(eps, L - n);"),
    ("threshold_strict", "if (dnorm >= thr * smax4[q]) sig = 1;", "if (dnorm > thr * smax4[q]) sig = 1;"),
    ("smax_floor", "    double m = 1.0;\n", "    double m = 0.0;\n"),
    ("threshold_without_bed", "for (int q = 0; q < 4; ++q) {\n        const double* d",
     "for (int q = 0; q < 3; ++q) {\n        const double* d"),
    ("detail_without_abs", "maxd(maxd(absd(d[0]), absd(d[1])), absd(d[2]))", "maxd(maxd(d[0], d[1]), d[2])"),
    ("predict_last_level", "for (int n = 0; n + 1 <= L - 1; ++n)", "for (int n = 0; n + 1 <= L - 2; ++n)"),
    ("predict_child_index", "2 * i + (k & 1), 2 * j + (k >> 1)", "2 * i + (k >> 1), 2 * j + (k >> 1)"),
    ("closure_transposed", "rm(n - 1, i / 2, j / 2)", "rm(n - 1, j / 2, i / 2)"),
    ("dft_child_order", "    dft_visit(ctx, n + 1, 2 * i + 1, 2 * j);\n    dft_visit(ctx, n + 1, 2 * i, 2 * j + 1);",
     "    dft_visit(ctx, n + 1, 2 * i, 2 * j + 1);\n    dft_visit(ctx, n + 1, 2 * i + 1, 2 * j);"),
    ("ptt_ancestor_shift", "uint64_t code = m >> (2 * (L - n));", "uint64_t code = m >> (L - n);"),
    ("reconstruction_min_bed", "double zf = maxd(zL, zR);", "double zf = zL < zR ? zL : zR;"),
    ("star_velocity_sign", "*us = 0.5 * (unL + unR) + aL - aR;", "*us = 0.5 * (unL + unR) + aR - aL;"),
    ("star_celerity_sign", "*as = 0.5 * (aL + aR) + 0.25 * (unL - unR);", "*as = 0.5 * (aL + aR) - 0.25 * (unL - unR);"),
    ("flux_pressure", "FL1 = qnL * unL + 0.5 * g * hLs * hLs", "FL1 = qnL * unL + g * hLs * hLs"),
    ("hll_jump_sign", "SL * SR * (hRs - hLs)", "SL * SR * (hLs - hRs)"),
    ("dry_left_speed", "SL = unR - 2.0 * aR;", "SL = unR - aR;"),
    ("dry_right_speed", "SR = unL + 2.0 * aL;", "SR = unL + aL;"),
    ("ghost_component", "if (s == ORC_W || s == ORC_E) c.qx = -c.qx;", "if (s == ORC_W || s == ORC_E) c.qy = -c.qy;"),
    ("bed_source_sign", "double bx = 0.5 * g * (hW2 - hE2);", "double bx = 0.5 * g * (hE2 - hW2);"),
    ("update_component", "double qx = C.qx - rx * ((FE[1] - FW[1]) + bx) - ry * (GN[2] - GS[2]);",
     "double qx = C.qx - rx * ((FE[1] - FW[1]) + bx) - ry * (GN[1] - GS[1]);"),
    ("no_positivity_clamp", "h = h > 0.0 ? h : 0.0;", "h = h;"),
    ("manning_exponent", "(h * cbrt(h))", "(h * sqrt(h))"),
    ("manning_n_squared", "dt * g * nM * nM * speed", "dt * g * nM * speed"),
    ("inflow_area", "return ((Q * dt) * frac) / (dx * dy);", "return ((Q * dt) * frac) / dx;"),
    ("hydrograph_weight", "(p->inflow_Q[k + 1] - p->inflow_Q[k]) * w", "(p->inflow_Q[k + 1] - p->inflow_Q[k]) * (1.0 - w)"),
    ("cfl_celerity", "    double a = sqrt(p->g * h);\n", "    double a = sqrt(h);\n"),
    ("cfl_number", "double dt = p->cfl * r;", "double dt = r;"),
    ("cfl_wet_cap", "return dt < p->dt_max ? dt : p->dt_max;", "return dt < INFINITY ? dt : p->dt_max;"),
    ("cfl_spacing", "double dx = ldexp(p->lx, -p->L), dy = ldexp(p->ly, -p->L);\n    double rh",
     "double dx = ldexp(p->lx, -p->L + 1), dy = ldexp(p->ly, -p->L + 1);\n    double rh"),
    ("decode_hands_down_depth", "int restore = n < L && hl >= p->tol_h;", "int restore = 0;"),
    ("decode_surface_bed", "double eta = restore ? hl + hier[3][level_start(n) + rm(n, i, j)] : 0.0;",
     "double eta = restore ? hl + z[rm(L, i * w, j * w)] : 0.0;"),
    ("leaf_spacing", "double dx = ldexp(p->lx, -n), dy = ldexp(p->ly, -n);",
     "double dx = ldexp(p->lx, -p->L), dy = ldexp(p->ly, -p->L);"),
    ("matched_depth_half", "*own2 = 0.5 * (oa + ob);", "*own2 = oa;"),
    ("matched_child", "cni = 2 * ni + (s == ORC_E ? 0 : 1);", "cni = 2 * ni + (s == ORC_E ? 1 : 0);"),
    ("uniform_neighbour", "orc_cell E = i < last ? CELL(i + 1, j)", "orc_cell E = i < last ? CELL(i, j + 1)"),
    # the learned subtree skip (R-skip)
    ("skip_storage_ignores_neighbours", "if (si > 0 && pred[rm(Ls, si - 1, sj)] > v) v = pred[rm(Ls, si - 1, sj)];",
     "if (0) v = pred[rm(Ls, si - 1, sj)];"),
    ("skip_encode_from_storage_level_only", "E[s] = P[s] > m[s] ? P[s] : m[s];", "E[s] = P[s];"),
    ("skip_leaf_clamp_off_by_one", "if (n >= pred[subtree_of(Ls, n, i, j)]) S[level_start(n) + rm(n, i, j)] = 0;",
     "if (n > pred[subtree_of(Ls, n, i, j)]) S[level_start(n) + rm(n, i, j)] = 0;"),
    ("skip_flags_below_prediction", "if (n >= Ls && n >= pred[subtree_of(Ls, n, i, j)]) continue;",
     "if (n >= Ls && n > pred[subtree_of(Ls, n, i, j)]) continue;"),
    ("skip_prolong_hands_down_depth", "            if (hl >= p->tol_h) {\n                double eta = hl + zh[ka];",
     "            if (0) {\n                double eta = hl + zh[ka];"),
    ("skip_store_bed_of_leaf_level", "                        double d = eta - zh[kc];\n                        hf = d > 0.0 ? d : 0.0;\n                    }\n                    hier3[0][kc] = hf;\n                    hier3[1][kc] = nv[1][kl];",
     "                        double d = eta - zh[kl];\n                        hf = d > 0.0 ? d : 0.0;\n                    }\n                    hier3[0][kc] = hf;\n                    hier3[1][kc] = nv[1][kl];"),
    ("skip_smax_without_floor", "smax3[0] = smax3[1] = smax3[2] = 1.0;", "smax3[0] = smax3[1] = smax3[2] = 0.0;"),
    ("skip_storage_level_not_updated", "for (int64_t s = 0; s < NSUB; ++s) m[s] = P[s];", "for (int64_t s = 0; s < NSUB; ++s) m[s] = m[s];"),
]


def _try(mutant, source):
    name, before, after = mutant
    d = os.path.join(WORK, name)
    shutil.rmtree(d, ignore_errors=True)
    os.makedirs(os.path.join(d, "_build"))
    src = os.path.join(d, "hwfv1_oracle.c")
    with open(src, "w") as fh:
        fh.write(source.replace(before, after))
    # it must build (a mutant that does not compile proves nothing)
    lib = os.path.join(d, "_build", "liborc_hwfv1.so")
    b = subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                        "-o", lib, src, "-lm"], capture_output=True, text=True)
    if b.returncode != 0:
        shutil.rmtree(d, ignore_errors=True)
        return name, "does not build: " + b.stderr[-300:]
    env = dict(os.environ, HWFV1_ORACLE_SRC=src, HWFV1_ORACLE_BUILD_DIR=os.path.join(d, "_build"))
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True)
    shutil.rmtree(d, ignore_errors=True)
    if r.returncode == 1:          # a pin failed
        return name, None
    return name, "survived (pytest exit %d)" % r.returncode


def test_every_planted_mistake_fails_a_pin():
    with open(SRC) as fh:
        source = fh.read()
    for name, before, _ in MUTANTS:
        assert source.count(before) == 1, "mutation site of %s not found once" % name
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(lambda m: _try(m, source), MUTANTS))
    bad = [(n, why) for n, why in res if why is not None]
    assert not bad, bad


# The CNN oracle (oracle/cnn.py, numpy): mutants run in this process against
# the pins of tests/test_oracle_cnn.py.
CNN_MUTANTS = [
    ("padding_offset", "    xp[:, :, 1:H + 1, 1:W + 1] = x\n    y = np.zeros", "    xp[:, :, 0:H, 0:W] = x\n    y = np.zeros"),
    ("convolution_not_correlation", 'y += np.einsum("oc,bchw->bohw", w[:, :, di, dj], patch)',
     'y += np.einsum("oc,bchw->bohw", w[:, :, 2 - di, 2 - dj], patch)'),
    ("no_bias", "y = np.zeros((B, w.shape[0], H, W)) + b[None, :, None, None]", "y = np.zeros((B, w.shape[0], H, W))"),
    ("no_first_relu", "a1 = rnd(np.maximum(z1, 0.0))", "a1 = rnd(z1)"),
    ("no_second_relu", "a2 = rnd(np.maximum(z2, 0.0))", "a2 = rnd(z2)"),
    ("softmax_over_all", "p = e / e.sum(axis=1, keepdims=True)", "p = e / e.sum()"),
    ("loss_per_image", "loss = -np.sum(onehot * np.log(p)) / npix", "loss = -np.sum(onehot * np.log(p)) / B"),
    ("dlogits_sign", "return loss, (p - onehot) / npix", "return loss, (onehot - p) / npix"),
    ("dlogits_per_image", "return loss, (p - onehot) / npix", "return loss, (p - onehot) / B"),
    ("no_second_relu_mask", "dz2 = rnd(da2 * (z2 > 0))", "dz2 = rnd(da2)"),
    ("no_first_relu_mask", "dz1 = rnd(da1 * (z1 > 0))", "dz1 = rnd(da1)"),
    ("weight_gradient_transposed", "            patch = xp[:, :, di:di + H, dj:dj + W]\n            dw[",
     "            patch = xp[:, :, dj:dj + H, di:di + W]\n            dw["),
    ("input_gradient_flipped", 'dxp[:, :, di:di + H, dj:dj + W] += np.einsum("oc,bohw->bchw", w[:, :, di, dj], dy)',
     'dxp[:, :, di:di + H, dj:dj + W] += np.einsum("oc,bohw->bchw", w[:, :, 2 - di, 2 - dj], dy)'),
    ("bias_gradient_scale", "db = dy.sum(axis=(0, 2, 3))", "db = dy.sum(axis=(0, 2, 3)) * 0.5"),
    ("layer_input_before_relu", "da1, dw2, db2 = conv3x3_backward(a1, w2, dz2)", "da1, dw2, db2 = conv3x3_backward(z1, w2, dz2)"),
    ("bf16_no_tie_to_even", "keep = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000", "keep = (f + 0x8000) & 0xFFFF0000"),
    ("bf16_truncates", "keep = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000", "keep = f & 0xFFFF0000"),
    ("bf16_hidden_gradient_not_rounded", "dz1 = rnd(da1 * (z1 > 0))", "dz1 = da1 * (z1 > 0)"),
    ("bf16_loss_gradient_not_rounded", "conv3x3_backward(a2, w3, rnd(dlogits))", "conv3x3_backward(a2, w3, dlogits)"),
    ("bf16_activation_not_rounded", "a2 = rnd(np.maximum(z2, 0.0))", "a2 = np.maximum(z2, 0.0)"),
]


def test_every_planted_mistake_in_the_cnn_oracle_fails_a_pin(monkeypatch):
    import types
    import test_oracle_cnn as pins
    with open(os.path.join(ROOT, "oracle", "cnn.py")) as fh:
        source = fh.read()
    checks = [getattr(pins, n) for n in sorted(dir(pins)) if n.startswith("test_")]
    survivors = []
    for name, before, after in CNN_MUTANTS:
        assert source.count(before) == 1, "mutation site of %s not found once" % name
        mod = types.ModuleType("cnn_mutant")
        exec(compile(source.replace(before, after), "cnn_mutant", "exec"), mod.__dict__)
        monkeypatch.setattr(pins, "cnn", mod)
        caught = False
        for check in checks:
            try:
                check()
            except AssertionError:
                caught = True
                break
        if not caught:
            survivors.append(name)
    assert not survivors, survivors
