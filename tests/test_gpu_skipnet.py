"""The subtree CNN on the tensor cores against its CPU oracle (forward values
and gradients), its training, the features and labels the simulation hands
it, and the learned look-ahead in the time loop."""
import numpy as np
import pytest

import oracle
import synth
from oracle import cnn

pytestmark = pytest.mark.gpu


def _bf16(a):
    import torch
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _flat(params):
    return np.concatenate([p.reshape(-1) for p in params]).astype(np.float32)


def _unflat(flat, like):
    out, k = [], 0
    for p in like:
        out.append(flat[k:k + p.size].reshape(p.shape).astype(np.float64))
        k += p.size
    return out


def _setup(seed, nimg=3, H=9, W=13):
    import torch
    from paper_2206_05761_gb300 import hwfv1 as Hh
    rng = np.random.default_rng(seed)
    params = cnn.init_params(rng)
    params[1] = 0.1 * rng.standard_normal(16)
    params[3] = 0.1 * rng.standard_normal(16)
    params[5] = 0.1 * rng.standard_normal(5)
    # the GPU holds bf16 weights and float32 biases: give the oracle the same values
    params = [_bf16(p) if p.ndim == 4 else p.astype(np.float32).astype(np.float64) for p in params]
    x = _bf16(rng.standard_normal((nimg, H, W, 4)))
    labels = rng.integers(0, 5, size=(nimg, H, W)).astype(np.uint8)
    net = Hh.hwfv1_skipnet_create(seed)
    Hh.hwfv1_skipnet_set_params(net, _flat(params))
    xd = torch.as_tensor(x.astype(np.float32)).to(torch.bfloat16).reshape(-1).cuda()
    ld = torch.as_tensor(labels).reshape(-1).cuda()
    return net, params, x, labels, xd, ld


# The network's stated precision is BF16 operands with FP32 accumulation;
# the oracle states the same network with its BF16 operands rounded where
# the network holds them (oracle/cnn.py) and everything else in float64.
# Element-wise bound against that oracle: every element of a forward output
# or gradient within 1e-2 of its oracle value, relative to |value| plus a
# tenth of the tensor's largest magnitude.  The floor is there because the
# two sides accumulate in different precisions (FP32 on the tensor cores,
# float64 here): where a hidden value lies next to a BF16 rounding boundary
# the two round it to neighbouring BF16 values (2^-8 apart relative), and
# that difference reaches the outputs near their zero crossings.  Against
# the plain float64 network (no operand rounding) the BF16 roundings
# themselves differ by up to 2^-9 per operand, so that comparison is held
# to a relative L2 error.
RTOL_BF16 = 1e-2
RL2_F64 = 5e-2


def _elementwise_err(got, ref):
    scale = np.abs(ref) + 0.1 * np.abs(ref).max()
    return float(np.max(np.abs(got - ref) / scale))


def _rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


SIZES = [(3, 9, 13), (2, 128, 128)]     # a ragged toy size and the production 128 x 128 image


@pytest.mark.parametrize("nimg,H,W", SIZES)
def test_forward_matches_oracle(nimg, H, W):
    import torch
    from paper_2206_05761_gb300 import hwfv1 as Hh
    net, params, x, labels, xd, _ = _setup(1, nimg, H, W)
    logits = torch.empty(nimg * H * W * 16, dtype=torch.float32, device="cuda")
    Hh.hwfv1_skipnet_forward(net, xd, nimg, H, W, logits)
    got = logits.cpu().numpy().reshape(nimg, H, W, 16)[..., :5].transpose(0, 3, 1, 2).astype(np.float64)
    xt = x.transpose(0, 3, 1, 2)
    e_bf = _elementwise_err(got, cnn.forward(params, xt, cnn.bf16)[0])
    r_64 = _rel_l2(got, cnn.forward(params, xt)[0])
    print("forward %dx%dx%d: element-wise error %.3g (BF16 operands), relative L2 %.3g (float64)"
          % (nimg, H, W, e_bf, r_64))
    assert e_bf <= RTOL_BF16 and r_64 <= RL2_F64
    Hh.hwfv1_skipnet_destroy(net)


@pytest.mark.parametrize("nimg,H,W", SIZES)
def test_gradients_match_oracle(nimg, H, W):
    from paper_2206_05761_gb300 import hwfv1 as Hh
    net, params, x, labels, xd, ld = _setup(2, nimg, H, W)
    loss, g = Hh.hwfv1_skipnet_gradients(net, xd, ld, nimg, H, W)
    got = _unflat(g, params)
    xt = x.transpose(0, 3, 1, 2)
    for tag, rnd in (("BF16 operands", cnn.bf16), ("float64", None)):
        logits, cache = cnn.forward(params, xt, rnd)
        ref_loss, dl = cnn.loss_and_dlogits(logits, labels)
        ref = cnn.backward(params, cache, dl, rnd)
        assert abs(loss - ref_loss) <= RTOL_BF16 * ref_loss
        for name, a, b in zip(("w1", "b1", "w2", "b2", "w3", "b3"), got, ref):
            if rnd is None:
                err = _rel_l2(a, b)
                print("gradient %s %dx%dx%d vs float64: relative L2 %.3g" % (name, nimg, H, W, err))
                assert err <= RL2_F64, (name, err)
            else:
                err = _elementwise_err(a, b)
                print("gradient %s %dx%dx%d vs BF16 operands: element-wise %.3g" % (name, nimg, H, W, err))
                assert err <= RTOL_BF16, (name, err)
    Hh.hwfv1_skipnet_destroy(net)


def test_training_reduces_loss():
    import torch
    from paper_2206_05761_gb300 import hwfv1 as Hh
    rng = np.random.default_rng(3)
    nimg, H, W = 64, 16, 16
    x = rng.standard_normal((nimg, H, W, 4)).astype(np.float32)
    # a label the network can learn: the level of a local average of channel 0
    sm = x[..., 0].copy()
    for _ in range(2):
        sm = (sm + np.roll(sm, 1, 1) + np.roll(sm, -1, 1) + np.roll(sm, 1, 2) + np.roll(sm, -1, 2)) / 5.0
    labels = np.clip(np.floor((sm / sm.std() + 2.5)), 0, 4).astype(np.uint8)
    xd = torch.as_tensor(x).to(torch.bfloat16).reshape(-1).cuda()
    ld = torch.as_tensor(labels).reshape(-1).cuda()
    net = Hh.hwfv1_skipnet_create(7)
    l0, _ = Hh.hwfv1_skipnet_gradients(net, xd, ld, nimg, H, W)
    Hh.hwfv1_skipnet_train(net, xd, ld, nimg, H, W, batch=8, epochs=40, lr=3e-3, seed=1)
    l1, _ = Hh.hwfv1_skipnet_gradients(net, xd, ld, nimg, H, W)
    print("training loss %.4f -> %.4f" % (l0, l1))
    assert l1 < 0.6 * l0
    Hh.hwfv1_skipnet_destroy(net)


def test_training_is_deterministic():
    # the backward pass sums in a fixed order (no float atomics): two networks
    # from one seed, trained on the same samples, end with the same bits
    import torch
    from paper_2206_05761_gb300 import hwfv1 as Hh
    rng = np.random.default_rng(5)
    nimg, H, W = 16, 32, 32
    x = torch.as_tensor(rng.standard_normal((nimg, H, W, 4)).astype(np.float32)).to(torch.bfloat16)
    labels = torch.as_tensor(rng.integers(0, 5, (nimg, H, W)).astype(np.uint8))
    xd, ld = x.reshape(-1).cuda(), labels.reshape(-1).cuda()
    out = []
    for _ in range(2):
        net = Hh.hwfv1_skipnet_create(11)
        Hh.hwfv1_skipnet_train(net, xd, ld, nimg, H, W, batch=4, epochs=3, lr=3e-3, seed=2)
        _, g = Hh.hwfv1_skipnet_gradients(net, xd, ld, nimg, H, W)
        out.append((Hh.hwfv1_skipnet_get_params(net), np.asarray(g)))
        Hh.hwfv1_skipnet_destroy(net)
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def _closure_labels(T, L):
    """Training labels from the oracle's threshold flags (row-major per level):
    close the flags upward and take, per level-(L-4) subtree, 1 + the deepest
    flagged level, minus (L-4)."""
    Ls = L - 4
    C = [None] * L
    for n in range(L - 1, -1, -1):
        s = 1 << n
        t = T[oracle.level_start(n): oracle.level_start(n) + s * s].reshape(s, s).astype(bool)
        if n + 1 < L:
            ch = C[n + 1]
            t = t | ch[0::2, 0::2] | ch[1::2, 0::2] | ch[0::2, 1::2] | ch[1::2, 1::2]
        C[n] = t
    S = 1 << Ls
    lab = np.zeros((S, S), np.uint8)
    for n in range(Ls, L):
        w = 1 << (n - Ls)
        blk = C[n].reshape(S, w, S, w).any(axis=(1, 3))
        lab[blk] = n + 1 - Ls
    return lab


def test_features_and_labels_match_oracle():
    import torch
    from paper_2206_05761_gb300.sim import Simulation
    L, Ls = 7, 3
    p, f = synth.bumpy_dam_break(L=L, eps=1e-3, seed=5)
    sim = Simulation(p, f)
    ref = oracle.State(p, f)
    for _ in range(4):
        sim.step()
        ref.step()
    # features: level-Ls scaling coefficients of the current state over s_max
    s = 1 << Ls
    exp = np.zeros((s, s, 4))
    for q, fine in enumerate((ref.h, ref.qx, ref.qy, ref.z)):
        hier, _ = oracle.encode(L, fine)
        exp[..., q] = oracle.level(hier, Ls) / oracle.smax(L, fine)
    exp_bf = torch.as_tensor(exp.astype(np.float32)).to(torch.bfloat16).float().numpy()
    res = ref.step(want=("T",))
    sim.encode()
    sim.flag()
    assert np.array_equal(sim.features(), exp_bf)
    assert np.array_equal(sim.labels(), _closure_labels(res["T"], L))
    sim.close()


@pytest.mark.parametrize("every", [1, 3])
def test_learned_mode_with_gate_open_equals_plain(every):
    from paper_2206_05761_gb300 import hwfv1 as Hh
    from paper_2206_05761_gb300.sim import Simulation
    p, f = synth.bumpy_dam_break(L=7, eps=1e-3, seed=6)
    a = Simulation(p, f)
    b = Simulation(p, f)
    net = Hh.hwfv1_skipnet_create(3)
    b.set_skipnet(net, audit_K=4, margin=-1.0, predict_every=every)
    a.advance(max_steps=15)
    b.advance(max_steps=15)
    ga, gb = a.fields(), b.fields()
    for k in ga:
        assert np.array_equal(ga[k], gb[k])
    assert np.array_equal(a.leaves(), b.leaves())
    a.close()
    b.close()
    Hh.hwfv1_skipnet_destroy(net)
