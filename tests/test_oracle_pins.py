"""Pins of the FP64 oracle against things other than itself (CPU only).

* closed forms of a single synapse's trace (Eq. filter, Eq. filtered-
  eligibility-trace) and the sum-of-Jacobian-products definition of the
  eligibility vector (Eq. eligibility-trace);
* hand-summed gradients of 1-neuron networks (LIF and ALIF);
* the autograd special case: BPTT through the network with the recurrent
  spike inputs and the reset term detached equals e-prop exactly
  (Eq. original-recurrent-weight-update with Eq. pdv_L_z);
* reductions (ALIF with beta_a = 0 is LIF; a batch of identical samples;
  parallel vs sequential mini-batches with reset);
* the event-driven restatement (Algorithm 5) equals the time-driven sum
  (Algorithm 1);
* the index flip (Eq. index-flipping): the future-facing sum equals the
  filtered, causal one.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.helpers import raster_to_lists, tau_for, tiny_net
from workloads import configs as C
from workloads import hashrng as H


# ---------------------------------------------------------------------------
# P1: closed forms of one synapse


def _run_synapse(alpha, rho, beta_a, kappa_e, psi, L, arrivals, T):
    st = np.zeros(3)
    g = 0.0
    ebars = []
    for t in range(1, T + 1):
        pp = psi[t - 2] if t >= 2 else 0.0
        g += oracle.eligibility_step(alpha, rho, beta_a, kappa_e, pp, psi[t - 1],
                                     L[t - 1], 1.0 if t in arrivals else 0.0, st)
        ebars.append(st[2])
    return g, np.asarray(ebars), st


def test_single_arrival_geometric_closed_form():
    # one arrival at a, constant psi = c and L = l:
    # ebar^t = c (kappa^{n+1} - alpha^{n+1}) / (kappa - alpha), n = t - a
    alpha, kappa, c, l, a, T = 0.9, 0.7, 0.35, -1.3, 4, 60
    g, ebars, _ = _run_synapse(alpha, 0.0, 0.0, kappa, [c] * T, [l] * T, {a}, T)
    n = np.arange(0, T - a + 1)
    expect = c * (kappa ** (n + 1) - alpha ** (n + 1)) / (kappa - alpha)
    np.testing.assert_allclose(ebars[a - 1:], expect, rtol=1e-13)
    assert np.all(ebars[:a - 1] == 0.0)
    Nn = T - a + 1
    G = l * c / (kappa - alpha) * (kappa * (1 - kappa ** Nn) / (1 - kappa)
                                   - alpha * (1 - alpha ** Nn) / (1 - alpha))
    assert g == pytest.approx(G, rel=1e-13)


def test_periodic_train_exact_rational():
    # presynaptic arrivals every p steps from s; constant psi, L; exact
    # rational double sums of the unrolled filters (Eq. filter)
    alpha, kappa, c, l = Fraction(1, 2), Fraction(3, 4), Fraction(2, 5), Fraction(-3, 7)
    p, s, T = 7, 3, 50
    arr = set(range(s, T + 1, p))
    zbar = [sum((alpha ** (t - a) for a in arr if a <= t), Fraction(0)) for t in range(1, T + 1)]
    ebar = [sum((kappa ** (t - u) * c * zbar[u - 1] for u in range(1, t + 1)), Fraction(0))
            for t in range(1, T + 1)]
    G = sum((l * e for e in ebar), Fraction(0))
    g, ebars, _ = _run_synapse(float(alpha), 0.0, 0.0, float(kappa), [float(c)] * T,
                               [float(l)] * T, arr, T)
    np.testing.assert_allclose(ebars, [float(e) for e in ebar], rtol=1e-13)
    assert g == pytest.approx(float(G), rel=1e-13)


def test_alif_vector_matches_jacobian_products():
    # Eq. eligibility-trace: eps^t = sum_{t'} (dh^t/dh^{t-1}) ... (dh^{t'+1}/dh^{t'}) dh^{t'}/dW
    rng = np.random.default_rng(3)
    T = 40
    alpha, rho, beta, kap = 0.93, 0.98, 1.7, 0.8
    psi = rng.uniform(0, 0.5, T)
    L = rng.normal(size=T)
    arrivals = {2, 5, 6, 13, 30}
    g, ebars, _ = _run_synapse(alpha, rho, beta, kap, psi, L, arrivals, T)

    def jac(t):  # dh^t/dh^{t-1}, h = (v, a); uses psi^{t-1}
        pp = psi[t - 2] if t >= 2 else 0.0
        return np.array([[alpha, 0.0], [pp, rho - pp * beta]])

    e = np.zeros(T)
    for t in range(1, T + 1):
        eps = np.zeros(2)
        for tp in range(1, t + 1):
            vec = np.array([1.0 if tp in arrivals else 0.0, 0.0])
            for u in range(tp + 1, t + 1):
                vec = jac(u) @ vec
            eps += vec
        e[t - 1] = psi[t - 1] * eps[0] - beta * psi[t - 1] * eps[1]
    ebar = np.zeros(T)
    acc = 0.0
    for t in range(T):
        acc = kap * acc + e[t]
        ebar[t] = acc
    np.testing.assert_allclose(ebars, ebar, rtol=1e-12, atol=1e-15)
    assert g == pytest.approx(float(np.dot(L, ebar)), rel=1e-12)


# ---------------------------------------------------------------------------
# P4: hand-summed 1-neuron networks (values worked out step by step)


def _hand_net(model, beta_a):
    net = tiny_net(1, 1, 1, [(0, 0)], [], [0.75], [], [1], [], [2.0],
                   dict(T=5, tau_m=tau_for(0.5), tau_out=tau_for(0.5),
                        tau_a=tau_for(0.5), neuron_model=model, beta_a=beta_a,
                        v_th=1.0, t_ref=0, gamma=0.5, beta_sg=1.0, lr=0.0,
                        max_delay=1))
    raster = np.zeros((1, 5, 1), bool)
    raster[0, [0, 1, 3], 0] = True           # input spikes emitted at t = 1, 2, 4
    x_ptr, x_ids = raster_to_lists(raster)
    o = oracle.Oracle(net["spec"], net["ptr"], net["col"], net["w"], net["delay"],
                      net["w_out"], net["out_mask"])
    r = o.simulate(5, x_ptr, x_ids, np.zeros((1, 5, 1)))
    return r, o.take_grads()


def test_hand_sum_lif():
    # w_in = 0.75, W_out = B = 2, alpha = kappa = 1/2, v_th = 1,
    # psi = 0.5 max(0, 1 - |v - 1|), input spikes emitted at 1, 2, 4 (arrive +1)
    # v: 0, 0.75, 1.125 (spike), -0.4375, 0.53125
    # psi: 0, 0.375, 0.4375, 0, 0.265625
    # y: 0, 0, 2, 1, 0.5 ; E = y ; L = 2 E = 0, 0, 4, 2, 1
    # zbar: 0, 1, 1.5, 0.75, 1.375
    # ebar: 0, 0.375, 0.84375, 0.421875, 0.576171875
    # g_in = 4*0.84375 + 2*0.421875 + 1*0.576171875 = 4.794921875
    # g_out = 2*1 + 1*0.5 + 0.5*0.25 = 2.625 ; loss = (4 + 1 + 0.25)/2
    r, (g, go) = _hand_net(0, 0.0)
    assert r["raster"][0, :, 0].tolist() == [0, 0, 1, 0, 0]
    np.testing.assert_array_equal(r["margin"][0, :, 0], [-1, -0.25, 0.125, -1.4375, -0.46875])
    np.testing.assert_array_equal(r["y"][0, :, 0], [0, 0, 2, 1, 0.5])
    assert r["loss"][0] == 2.625
    assert g[0] == 4.794921875
    assert go[0, 0] == 2.625


def test_hand_sum_alif():
    # as above with rho = 1/2, beta_a = 1:
    # a: 0, 0, 0, 1, 0.5 ; v_th: 1, 1, 1, 2, 1.5
    # v: 0, 0.75, 1.125 (spike), -1.4375, 0.03125 ; psi: 0, 0.375, 0.4375, 0, 0
    # eps_a: 0, 0, 0.375, 0.6796875, 0.33984375
    # e: 0, 0.375, 0.4375*(1.5-0.375) = 0.4921875, 0, 0
    # ebar: 0, 0.375, 0.6796875, 0.33984375, 0.169921875
    # g_in = 4*0.6796875 + 2*0.33984375 + 1*0.169921875 = 3.568359375
    r, (g, go) = _hand_net(1, 1.0)
    assert r["raster"][0, :, 0].tolist() == [0, 0, 1, 0, 0]
    np.testing.assert_array_equal(r["margin"][0, :, 0], [-1, -0.25, 0.125, -3.4375, -1.46875])
    assert g[0] == 3.568359375
    assert go[0, 0] == 2.625


# ---------------------------------------------------------------------------
# P2: BPTT with stop-gradients equals e-prop


torch = pytest.importorskip("torch")


class _Spike(torch.autograd.Function):
    """Heaviside forward (values given), surrogate psi backward: piecewise
    linear (Eq. piecewise-linear-surrogate-gradient) or exponential
    (Eq. exponential-surrogate-gradient)."""

    @staticmethod
    def forward(ctx, m, z_given, refr, gamma, beta, kind=0):
        ctx.save_for_backward(m, refr)
        ctx.gamma, ctx.beta, ctx.kind = gamma, beta, kind
        return z_given.clone()

    @staticmethod
    def backward(ctx, gz):
        m, refr = ctx.saved_tensors
        if ctx.kind == 1:
            psi = ctx.gamma * torch.exp(-ctx.beta * m.abs()) * (~refr)
        else:
            psi = ctx.gamma * torch.clamp(1.0 - ctx.beta * m.abs(), min=0.0) * (~refr)
        return gz * psi, None, None, None, None, None


def _bptt(net, T, x_raster, targets, window, lengths, z_raster):
    """Autograd gradient of the batch-mean loss; recurrent spike inputs and
    the reset term are detached, the neuron's own adaptation path is not.
    Variants of the spec: exponential surrogate, fixed reset (the whole
    reset correction detached), temporal MSE, and the firing-rate
    regularisation loss (c_reg / 2) sum_t sum_j (f_j^t - f*)^2 with the
    exponential moving average rate (Eq. ema-rate)."""
    s = net["spec"]
    B, N, K, NI = s.batch, s.n_rec, s.n_out, s.n_in
    # the parameter values as the oracle (and the library) take them
    pv = oracle.params(s)
    alpha, rho, kappa, beta_a = pv["alpha"], pv["rho"], pv["kappa"], pv["beta_a"]
    v_th, gamma, beta_sg, v_reset = pv["v_th"], pv["gamma"], pv["beta_sg"], pv["v_reset"]
    c_reg, f_target, beta_reg = pv["c_reg"], pv["f_target"], pv["beta_reg"]
    ptr = net["ptr"]
    src = torch.tensor(np.repeat(np.arange(len(ptr) - 1), np.diff(ptr)))
    col = torch.tensor(net["col"].astype(np.int64))
    dly = torch.tensor(net["delay"].astype(np.int64))
    w = torch.tensor(net["w"].astype(np.float64), requires_grad=True)
    wo = torch.tensor(net["w_out"].astype(np.float64), requires_grad=True)
    # generalized delays: the readout sees z^{t - d_out}; the recurrent and
    # input weights learn from the loss terms whose learning signal arrives
    # within the sample (t <= length - d_ls), the readout from all of them
    d_out, d_ls = int(getattr(s, "d_out", 0)), int(getattr(s, "d_ls", 0))
    total = 0.0
    total_rec = 0.0
    for b in range(B):
        v = torch.zeros(N, dtype=torch.float64)
        a = torch.zeros(N, dtype=torch.float64)
        zprev = torch.zeros(N, dtype=torch.float64)
        f = torch.zeros(N, dtype=torch.float64)
        ref = np.zeros(N, dtype=np.int64)
        y = torch.zeros(K, dtype=torch.float64)
        hist = {}
        zs = {}
        for t in range(1, int(lengths[b]) + 1):
            arrive = torch.zeros(len(src), dtype=torch.float64)
            for q in range(len(src)):
                tt = t - int(dly[q])
                if tt >= 1:
                    arrive[q] = hist[tt][int(src[q])]
            I = torch.zeros(N, dtype=torch.float64).index_add(0, col, w * arrive)
            a = rho * a + zprev
            vth = v_th + beta_a * a
            if s.reset_mode == 1:
                v = alpha * v + I + (zprev * (v_reset - alpha * v)).detach()
            else:
                v = alpha * v + I - (zprev * vth).detach()
            refr = torch.tensor(ref > 0)
            zg = torch.tensor(z_raster[b, t - 1].astype(np.float64))
            z = _Spike.apply(v - vth, zg, refr, gamma, beta_sg, s.surrogate)
            ref = np.where(ref > 0, ref - 1, 0)
            ref[z_raster[b, t - 1] > 0] = s.t_ref
            hist[t] = torch.cat([torch.tensor(x_raster[b, t - 1].astype(np.float64)),
                                 z.detach()])
            zs[t] = z
            zd = zs[t - d_out] if t - d_out >= 1 else torch.zeros(N, dtype=torch.float64)
            y = kappa * y + zd @ wo
            win = float(window[b, t - 1])
            tg = torch.tensor(targets[b, t - 1].astype(np.float64))
            if s.loss == 0:
                term = 0.5 * win * ((y - tg) ** 2).sum()
            elif s.loss == 2:
                term = win * ((y - tg) ** 2).sum() / K
            else:
                term = -win * (tg * torch.log_softmax(y, 0)).sum()
            total = total + term
            if t <= int(lengths[b]) - d_ls:
                total_rec = total_rec + term
            if c_reg != 0.0:
                f = beta_reg * f + (1.0 - beta_reg) * z
                reg = 0.5 * c_reg * ((f - f_target) ** 2).sum()
                total = total + reg
                total_rec = total_rec + reg
            zprev = z
    if d_out == 0 and d_ls == 0:
        (total / B).backward()
        return w.grad.numpy(), wo.grad.numpy()
    gw = torch.autograd.grad(total_rec / B, w, retain_graph=True, allow_unused=True)[0]
    gwo = torch.autograd.grad(total / B, wo)[0]
    gw = torch.zeros_like(w) if gw is None else gw
    return gw.numpy(), gwo.numpy()


def _random_small(model, loss, seed, B=2, T=40, n_in=3, N=6, K=2, max_delay=3):
    rng = np.random.default_rng(seed)
    pairs_in = [(i, j) for i in range(n_in) for j in range(N)]
    pairs_rec = [(i, j) for i in range(N) for j in range(N) if i != j]
    w_in = rng.normal(0.3, 1.0, len(pairs_in))
    w_rec = rng.normal(0, 0.5, len(pairs_rec))
    d_in = rng.integers(1, max_delay + 1, len(pairs_in))
    d_rec = rng.integers(1, max_delay + 1, len(pairs_rec))
    net = tiny_net(n_in, N, K, pairs_in, pairs_rec, w_in, w_rec, d_in, d_rec,
                   rng.normal(0, 0.5, (N, K)),
                   dict(batch=B, T=T, neuron_model=model,
                        beta_a=1.7 if model else 0.0, tau_a=30.0, loss=loss,
                        max_delay=max_delay, lr=0.0, t_ref=2))
    x = rng.random((B, T, n_in)) < 0.3
    if loss == 0:
        tg = rng.normal(size=(B, T, K))
    else:
        tg = np.zeros((B, T, K))
        tg[np.arange(B), :, rng.integers(0, K, B)] = 1.0
    lengths = np.array([T - 7 * b for b in range(B)], np.int32)
    window = np.ones((B, T), np.uint8)
    if loss >= 1:
        window[:] = 0
        for b in range(B):
            window[b, lengths[b] - 10:lengths[b]] = 1
    return net, x, tg, window, lengths


# e-prop+ variants, each alone: exponential surrogate, fixed reset, temporal
# MSE, firing-rate regularisation (Eq. ema-gradient)
VARIANTS = {
    "plain": {},
    "exp_surrogate": dict(surrogate=1),
    "fixed_reset": dict(reset_mode=1, v_reset=0.15),
    "rate_reg": dict(c_reg=3.0, f_target=0.05, beta_reg=0.9),
}


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("model,loss", [(0, 0), (1, 0), (0, 1), (1, 1), (0, 2), (1, 2)])
def test_eprop_equals_bptt_with_stop_gradients(model, loss, variant):
    if loss == 2 and variant != "plain":
        pytest.skip("temporal MSE is checked with the plain neuron")
    net, x, tg, window, lengths = _random_small(model, loss, seed=10 + 2 * model + min(loss, 1))
    s = net["spec"]
    for k, v in VARIANTS[variant].items():
        setattr(s, k, v)
    o = oracle.Oracle(s, net["ptr"], net["col"], net["w"], net["delay"], net["w_out"],
                      net["out_mask"])
    x_ptr, x_ids = raster_to_lists(x)
    r = o.simulate(s.T, x_ptr, x_ids, tg, window, lengths)
    assert r["raster"].sum() > 5, "test network must spike"
    g, go = o.take_grads()
    gw, gwo = _bptt(net, s.T, x, tg, window, lengths, r["raster"])
    scale = np.abs(gw).max()
    np.testing.assert_allclose(g, gw, rtol=1e-9, atol=1e-12 * scale)
    np.testing.assert_allclose(go, gwo, rtol=1e-9, atol=1e-12 * np.abs(gwo).max())


@pytest.mark.parametrize("d_out,d_ls", [(1, 0), (0, 2), (2, 3)])
@pytest.mark.parametrize("model,loss", [(0, 0), (1, 1)])
def test_generalized_delays_equal_bptt(model, loss, d_out, d_ls):
    # Supplement "Generalized delays": the readout sees the recurrent spikes
    # d_out steps late and the learning signal reaches the recurrent layer
    # d_ls steps late; e-prop pairs L^tau with the eligibility of tau - d_out
    # and drops the signals that arrive after the sample's end
    net, x, tg, window, lengths = _random_small(model, loss, seed=30 + 2 * model + loss + d_out)
    s = net["spec"]
    s.d_out, s.d_ls = d_out, d_ls
    o = oracle.Oracle(s, net["ptr"], net["col"], net["w"], net["delay"], net["w_out"],
                      net["out_mask"])
    x_ptr, x_ids = raster_to_lists(x)
    r = o.simulate(s.T, x_ptr, x_ids, tg, window, lengths)
    assert r["raster"].sum() > 5, "test network must spike"
    g, go = o.take_grads()
    gw, gwo = _bptt(net, s.T, x, tg, window, lengths, r["raster"])
    scale = np.abs(gw).max()
    assert scale > 0
    np.testing.assert_allclose(g, gw, rtol=1e-9, atol=1e-12 * scale)
    np.testing.assert_allclose(go, gwo, rtol=1e-9, atol=1e-12 * np.abs(gwo).max())
    # the delays change the gradient (the pin is not the undelayed one)
    s.d_out, s.d_ls = 0, 0
    g0, _ = _bptt(net, s.T, x, tg, window, lengths, r["raster"])
    assert np.abs(g0 - gw).max() > 1e-6 * scale


# ---------------------------------------------------------------------------
# P5: reductions


def _cfg0_small(**kw):
    W = C.pattern_regression(T=200, n_rec=30, n_in=10, **kw)
    return W


def _run(W, **spec_over):
    s = W["spec"]
    for k, v in spec_over.items():
        setattr(s, k, v)
    o = oracle.Oracle(s, W["ptr"], W["col"], W["w"], W["delay"], W["w_out"], W["out_mask"],
                      W["feedback"])
    r = o.simulate(s.T, W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"])
    return r, o.take_grads(), o


def test_alif_with_zero_adaptation_is_lif():
    r1, (g1, go1), _ = _run(_cfg0_small(), neuron_model=0)
    r2, (g2, go2), _ = _run(_cfg0_small(), neuron_model=1, beta_a=0.0)
    assert np.array_equal(r1["raster"], r2["raster"])
    assert np.array_equal(g1, g2) and np.array_equal(go1, go2)


def test_batch_of_identical_samples_equals_single():
    W1 = _cfg0_small()
    r1, (g1, go1), _ = _run(W1)
    W2 = _cfg0_small()
    B = 3
    W2["spec"].batch = B
    T = W2["spec"].T
    ptr, ids = W1["x_ptr"], W1["x_ids"]
    W2["x_ptr"] = np.concatenate([[0]] + [ptr[1:] + b * ptr[-1] for b in range(B)])
    W2["x_ids"] = np.tile(ids, B)
    W2["targets"] = np.repeat(W1["targets"], B, axis=0)
    W2["window"] = np.ones((B, T), np.uint8)
    W2["lengths"] = np.full(B, T, np.int32)
    r2, (g2, go2), _ = _run(W2)
    for b in range(B):
        assert np.array_equal(r2["raster"][b], r1["raster"][0])
    np.testing.assert_allclose(g2, g1, rtol=1e-13, atol=1e-13 * np.abs(g1).max())
    np.testing.assert_allclose(go2, go1, rtol=1e-13, atol=1e-13 * np.abs(go1).max())


def test_parallel_equals_sequential_minibatch_with_reset():
    # batch of two different samples vs the two samples one by one (lr = 0)
    rng = np.random.default_rng(5)
    W = _cfg0_small(batch=2)
    T = W["spec"].T
    raster = rng.random((2, T, W["spec"].n_in)) < 0.05
    W["x_ptr"], W["x_ids"] = raster_to_lists(raster)
    W["targets"] = rng.normal(size=(2, T, 1)).astype(np.float32)
    W["window"] = np.ones((2, T), np.uint8)
    W["lengths"] = np.array([T, T - 30], np.int32)
    W["spec"].lr = 0.0
    rb, (gb, gob), _ = _run(W)
    gs, gos = [], []
    for b in range(2):
        Wb = _cfg0_small()
        Wb["spec"].lr = 0.0
        Wb["x_ptr"], Wb["x_ids"] = raster_to_lists(raster[b:b + 1])
        Wb["targets"] = W["targets"][b:b + 1]
        Wb["lengths"] = W["lengths"][b:b + 1]
        r, (g, go), _ = _run(Wb)
        assert np.array_equal(r["raster"][0, :W["lengths"][b]], rb["raster"][b, :W["lengths"][b]])
        gs.append(g)
        gos.append(go)
    np.testing.assert_allclose(gb, (gs[0] + gs[1]) / 2, rtol=1e-12, atol=1e-12 * np.abs(gb).max())
    np.testing.assert_allclose(gob, (gos[0] + gos[1]) / 2, rtol=1e-12,
                               atol=1e-12 * np.abs(gob).max())


# ---------------------------------------------------------------------------
# P3: event-driven organisation equals time-driven


def _source_raster(spec, x_ptr, x_ids, raster_rec, b, T):
    src = np.zeros((T, spec.n_in + spec.n_rec), np.uint8)
    for t in range(T):
        q = b * T + t
        src[t, x_ids[x_ptr[q]:x_ptr[q + 1]]] = 1
    src[:, spec.n_in:] = raster_rec[b]
    return src


@pytest.mark.parametrize("model", [0, 1])
def test_event_driven_equals_time_driven(model):
    net, x, tg, window, lengths = _random_small(model, 0, seed=40 + model, B=1, T=60,
                                                max_delay=4)
    s = net["spec"]
    o = oracle.Oracle(s, net["ptr"], net["col"], net["w"], net["delay"], net["w_out"],
                      net["out_mask"])
    x_ptr, x_ids = raster_to_lists(x)
    r = o.simulate(s.T, x_ptr, x_ids, tg, window, lengths, record=True)
    g, _ = o.take_grads()
    src = _source_raster(s, x_ptr, x_ids, r["raster"], 0, s.T)
    ge = oracle.event_driven_gradients(s, net["ptr"], net["col"], net["delay"], src,
                                       r["psi"][0], r["L"][0], int(lengths[0]))
    np.testing.assert_allclose(ge, g, rtol=1e-12, atol=1e-12 * np.abs(g).max())


@pytest.mark.parametrize("model", [0, 1])
def test_arrival_contributions_sum_to_the_gradient(model):
    # linearity of the eligibility recursion in the presynaptic trace: the
    # time-driven gradient of a synapse equals the sum, over its arrivals a,
    # of the forward response Q_j(a) to one unit arrival at a (the per-event
    # term of the event-driven update); |.| summed bounds |g| from above
    net, x, tg, window, lengths = _random_small(model, 0, seed=50 + model, B=1, T=60,
                                                max_delay=4)
    s = net["spec"]
    o = oracle.Oracle(s, net["ptr"], net["col"], net["w"], net["delay"], net["w_out"],
                      net["out_mask"])
    x_ptr, x_ids = raster_to_lists(x)
    r = o.simulate(s.T, x_ptr, x_ids, tg, window, lengths, record=True)
    g, _ = o.take_grads()
    Q = oracle.arrival_contrib(s, r["psi"][0], r["L"][0])
    src = _source_raster(s, x_ptr, x_ids, r["raster"], 0, s.T)
    ge = np.zeros_like(g)
    for i in range(src.shape[1]):
        for st in np.nonzero(src[:, i])[0] + 1:
            for q in range(int(net["ptr"][i]), int(net["ptr"][i + 1])):
                a = int(st) + int(net["delay"][q])
                if a <= s.T:
                    ge[q] += Q[a - 1, int(net["col"][q])]
    assert np.abs(g).max() > 0
    np.testing.assert_allclose(ge, g, rtol=1e-12, atol=1e-12 * np.abs(g).max())
    mag = oracle.arrival_magnitude(s, net["ptr"], net["col"], net["delay"], x_ptr, x_ids,
                                   lengths, r["raster"], r["psi"], r["L"])
    assert np.all(mag >= np.abs(g) * (1 - 1e-12))


@pytest.mark.parametrize("model", [0, 1])
def test_error_override_with_the_true_signal_is_the_full_window_run(model):
    # the override replaces E only where the window is closed: feeding it the
    # error signal of a run with the window open everywhere, and closing the
    # window, must reproduce that run's gradients and readout gradients
    net, x, tg, window, lengths = _random_small(model, 1, seed=60 + model)
    s = net["spec"]
    x_ptr, x_ids = raster_to_lists(x)
    args = (net["ptr"], net["col"], net["w"], net["delay"], net["w_out"], net["out_mask"])
    o1 = oracle.Oracle(s, *args)
    ones = np.ones_like(window)
    r1 = o1.simulate(s.T, x_ptr, x_ids, tg, ones, lengths)
    g1, go1 = o1.take_grads()
    y = r1["y"]
    E = np.exp(y - y.max(axis=2, keepdims=True))
    E = E / E.sum(axis=2, keepdims=True) - tg
    o2 = oracle.Oracle(s, *args)
    o2.simulate(s.T, x_ptr, x_ids, tg, np.zeros_like(window), lengths, E_override=E)
    g2, go2 = o2.take_grads()
    assert np.abs(g1).max() > 0
    np.testing.assert_allclose(g2, g1, rtol=1e-12, atol=1e-13 * np.abs(g1).max())
    np.testing.assert_allclose(go2, go1, rtol=1e-12, atol=1e-13 * np.abs(go1).max())
    # with the window open the override is ignored
    o3 = oracle.Oracle(s, *args)
    o3.simulate(s.T, x_ptr, x_ids, tg, ones, lengths, E_override=np.full_like(E, 7.0))
    g3, _ = o3.take_grads()
    np.testing.assert_array_equal(g3, g1)


def test_index_flip_future_facing_form():
    # Eq. summation-future: sum_{t'} dL/dz^{t'} e^{t'}, with dL/dz^{t'} =
    # sum_k B_jk sum_{t >= t'} kappa^{t - t'} E_k^t, equals the oracle's causal
    # sum_t L^t F_kappa(e^t) (LIF, d = 1: e^t = psi^t F_alpha(z_i^{t-1})).
    net, x, tg, window, lengths = _random_small(0, 0, seed=77, B=1, T=50, max_delay=1)
    s = net["spec"]
    o = oracle.Oracle(s, net["ptr"], net["col"], net["w"], net["delay"], net["w_out"],
                      net["out_mask"])
    x_ptr, x_ids = raster_to_lists(x)
    r = o.simulate(s.T, x_ptr, x_ids, tg, window, lengths, record=True)
    g, _ = o.take_grads()
    T = int(lengths[0])
    alpha, kappa = math.exp(-1 / s.tau_m), math.exp(-1 / s.tau_out)
    src = _source_raster(s, x_ptr, x_ids, r["raster"], 0, s.T)
    psi, L = r["psi"][0], r["L"][0]
    ptr = net["ptr"]
    expect = np.zeros_like(g)
    for i in range(len(ptr) - 1):
        for q in range(ptr[i], ptr[i + 1]):
            j = net["col"][q]
            zbar, e = 0.0, np.zeros(T)
            for t in range(1, T + 1):
                zbar = alpha * zbar + (src[t - 2, i] if t >= 2 else 0)
                e[t - 1] = psi[t - 1, j] * zbar
            tot = 0.0
            for tp in range(1, T + 1):
                fut = sum(kappa ** (t - tp) * L[t - 1, j] for t in range(tp, T + 1))
                tot += fut * e[tp - 1]
            expect[q] = tot
    np.testing.assert_allclose(g, expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())


# ---------------------------------------------------------------------------
# drive: the oracle's counter hash reproduces the generator's definition


def test_drive_counts_follow_splitmix_definition():
    net = tiny_net(0, 3, 1, [], [], [], [], [], [], np.zeros((3, 1)),
                   dict(T=50, v_th=1e9, t_ref=0, drive_weight=0.25, drive_rate=1.5,
                        drive_seed=987654321, lr=0.0, max_delay=1))
    s = net["spec"]
    o = oracle.Oracle(s, net["ptr"], net["col"], net["w"], net["delay"], net["w_out"],
                      net["out_mask"])
    r = o.simulate(50, np.zeros(51, np.int64), np.zeros(0, np.int32), np.zeros((1, 50, 1)))
    v = r["margin"][0] + s.v_th
    alpha = math.exp(-1 / s.tau_m)
    vprev = np.vstack([np.zeros((1, 3)), v[:-1]])
    counts = np.rint((v - alpha * vprev) / s.drive_weight).astype(int)
    thr = s.drive_thresholds()
    for t in range(1, 51):
        for j in range(3):
            u = H.drive_hash_int(s.drive_seed, 0, t, j) >> 32
            assert counts[t - 1, j] == int(np.sum(u >= thr))
    assert counts.mean() == pytest.approx(1.5, abs=0.4)


def test_splitmix_reference_vector():
    # first outputs of SplitMix64 seeded with 0 (published reference values)
    assert H.mix_int(0) == 0xE220A8397B1DCDAF
    assert H.mix_int(H.GOLDEN) == 0x6E789E6AA1B965F4
    assert H.mix_int((2 * H.GOLDEN) % (1 << 64)) == 0x06C45D188009454F
