"""Learned closure on the GPU against the FP64 reference (oracle/closure.py):
restriction, MLP forward, backward (gradient) and the conserving correction;
then a small end-to-end training run that must lower the low-order error."""

import numpy as np
import pytest

import oracle
from oracle import closure as C
from paper_1612_01287_gb300 import workloads

pytestmark = pytest.mark.gpu

QL, QLO, QHI = 3, 8, 200
V = QL * QLO
D, H, O = 3 * V + 1, 64, V


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01287_gb300 import build, load
    build.build()
    load()


def sod_pair(Z, tau, dt, fields=None, bc="outflow"):
    from paper_1612_01287_gb300 import Sod
    kw = dict(Z=Z, Q_L=QL, N_Omega=5, precision="f32", bc=bc, tau=tau, dt=dt)
    if fields is not None:
        kw["fields"] = fields
    return Sod(Q_xi=QHI, **kw), Sod(Q_xi=QLO, **kw)


def oracle_theta(theta):
    """The parameters as the GPU uses them: BF16 weights, FP32 biases."""
    s = C.param_sizes(D, H, O)
    out, o = [], 0
    for k, n in enumerate(s):
        part = np.asarray(theta[o:o + n], dtype=np.float32)
        out.append(C.bf16_round(part) if k % 2 == 0 else part.astype(np.float64))
        o += n
    return np.concatenate(out)


def test_restriction_matches_oracle():
    from paper_1612_01287_gb300 import restrict
    Z = 96
    n, T, b = workloads.random_smooth_fields(Z, beta_max=0.5)
    hi, lo = sod_pair(Z, 0.05, 1e-3, fields=(n, T, b))
    with hi, lo:
        hi.step(5)
        fh = hi.get_state().astype(np.float64).T  # [Z][V_hi]
        restrict(hi, lo)
        fl = lo.get_state().astype(np.float64).T
    ref = C.restrict(fh, QHI, QLO, QL)
    assert np.abs(fl - ref).max() <= 2e-6 * np.abs(ref).max()


def random_norm(rng):
    mu = rng.normal(0, 0.5, size=D).astype(np.float32)
    isd = rng.uniform(0.5, 3.0, size=D).astype(np.float32)
    osd = rng.uniform(1e-3, 1e-1, size=O).astype(np.float32)
    return mu, isd, osd


def f64(norm):
    return tuple(np.asarray(a, dtype=np.float64) for a in norm)


def test_mlp_forward_matches_oracle():
    import torch
    from paper_1612_01287_gb300 import MLP
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, size=(300, D)).astype(np.float32)
    norm = random_norm(rng)
    with MLP(D, H, O, seed=7) as m:
        m.set_normalization(*norm)
        back = m.get_normalization()
        assert all(np.array_equal(a, b) for a, b in zip(back, norm))
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.zeros((300, O), dtype=torch.float32, device="cuda")
        m.forward(Xd.data_ptr(), 300, Yd.data_ptr())
        torch.cuda.synchronize()
        th = oracle_theta(m.get_params())
    ref = C.net(th, X.astype(np.float64), D, H, O, f64(norm))
    got = Yd.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_fit_normalization_matches_column_statistics():
    import torch
    from paper_1612_01287_gb300 import MLP
    rng = np.random.default_rng(6)
    X = rng.normal(2.0, 0.3, size=(20000, D)).astype(np.float32)
    X[:, -1] = -1.0  # a constant column (log10 tau of a single run)
    T = rng.normal(0, 1e-4, size=(20000, O)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()  # kept alive
    with MLP(D, H, O, seed=1) as m:
        m.fit_normalization(Xd.data_ptr(), Td.data_ptr(), 20000)
        mu, isd, osd = m.get_normalization()
    rmu, risd, rosd = C.fit_normalization(X, T)
    assert np.abs(mu - rmu).max() <= 1e-6 * np.abs(rmu).max()
    assert np.abs(isd - risd).max() <= 1e-5 * np.abs(risd).max()
    assert np.abs(osd - rosd).max() <= 1e-5 * np.abs(rosd).max()
    assert isd[-1] == 1.0


def test_mlp_gradient_matches_oracle():
    """Backward kernels vs FP64 backprop (all parameters) and vs the oracle's
    central differences on 1000 random parameters: relative error <= 1e-3."""
    import torch
    from paper_1612_01287_gb300 import MLP
    rng = np.random.default_rng(2)
    N = 256
    X = rng.normal(0, 1, size=(N, D)).astype(np.float32)
    T = rng.normal(0, 0.1, size=(N, O)).astype(np.float32)
    norm = random_norm(rng)
    with MLP(D, H, O, seed=3) as m:
        theta = m.get_params()
        theta[-O:] = rng.normal(0, 0.1, size=O)  # non-zero output biases
        theta[D * H:D * H + H] = rng.normal(0, 0.1, size=H)
        m.set_params(theta)
        m.set_normalization(*norm)
        Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        loss, g = m.loss_grad(Xd.data_ptr(), Td.data_ptr(), N)
        th = oracle_theta(m.get_params())
    mu, isd, osd = f64(norm)
    Xn = (X.astype(np.float64) - mu) * isd
    Tn = T.astype(np.float64) / osd
    Lr, gr = C.loss_grad(th, Xn, Tn, D, H, O)
    assert abs(loss - Lr) <= 1e-5 * Lr
    rel = np.abs(g - gr).max() / np.abs(gr).max()
    print("gradient vs FP64 backprop:", rel)
    assert rel <= 1e-3
    idx = rng.choice(len(th), size=1000, replace=False)
    fd = C.fd_grad(th, Xn, Tn, D, H, O, idx, h=1e-4)
    rel_fd = np.abs(g[idx] - fd).max() / np.abs(fd).max()
    print("gradient vs oracle finite differences:", rel_fd)
    assert rel_fd <= 1e-3


def test_closure_sample_matches_oracle():
    import torch
    from paper_1612_01287_gb300 import closure_sample
    Z, tau, dt = 64, 0.02, 2e-3
    n, T0, b = workloads.random_smooth_fields(Z, beta_max=0.4)
    hi, lo = sod_pair(Z, tau, dt, fields=(n, T0, b))
    with hi, lo:
        hi.step(3)
        f0 = hi.get_state().astype(np.float64).T
        Xd = torch.zeros((Z, D), device="cuda")
        Td = torch.zeros((Z, O), device="cuda")
        closure_sample(hi, lo, tau, Xd.data_ptr(), Td.data_ptr())
        X, T = Xd.cpu().numpy(), Td.cpu().numpy()
    r0 = C.restrict(f0, QHI, QLO, QL)
    assert np.abs(X - C.features(r0, tau)).max() <= 2e-6 * np.abs(X[:, :-1]).max()
    ph = oracle.sod_params(Z, QHI, QL, 5, bc="outflow", tau=tau, dt=dt)
    pl = oracle.sod_params(Z, QLO, QL, 5, bc="outflow", tau=tau, dt=dt)
    f1 = oracle.sod_steps(ph, f0, 1)
    pred = oracle.sod_steps(pl, r0, 1)
    Tref = C.project(C.restrict(f1, QHI, QLO, QL) - pred, QLO, QL) / r0.sum(1)[:, None]
    scale = np.abs(r0).max() / r0.sum(1).min()
    assert np.abs(T - Tref).max() <= 2e-6 * scale


def test_closure_step_matches_oracle_and_conserves():
    from paper_1612_01287_gb300 import MLP, Sod, closure_step
    Z, tau, dt = 80, 0.05, 2e-3
    n, T0, b = workloads.random_smooth_fields(Z, beta_max=0.4)
    kw = dict(Z=Z, Q_xi=QLO, Q_L=QL, N_Omega=5, precision="f32", bc="outflow", tau=tau, dt=dt,
              fields=(n, T0, b))
    rng = np.random.default_rng(12)
    norm = random_norm(rng)
    with MLP(D, H, O, seed=5) as m, Sod(**kw) as a, Sod(**kw) as c:
        th = m.get_params()
        th[D * H + H + H * H + H:] *= 10.0  # a visible correction
        m.set_params(th)
        m.set_normalization(*norm)
        a.step(1)
        closure_step(c, m, tau, 1)
        fa = a.get_state().astype(np.float64).T
        fc = c.get_state().astype(np.float64).T
        thr = oracle_theta(m.get_params())
    d = fc - fa
    ref = C.correction(thr, fa, tau, QLO, QL, H, f64(norm))
    assert np.abs(ref).max() > 1e-4 * np.abs(fa).max()
    assert np.abs(d - ref).max() <= 1e-5 * np.abs(fa).max()
    Phi, _ = C.invariants(QLO, QL)
    inv_a, inv_c = fa @ Phi, fc @ Phi
    assert np.abs(inv_c - inv_a).max() <= 2e-6 * np.abs(inv_a).max()


def test_closure_step_at_full_size_matches_oracle():
    """The correction of one closure step at 65536 cells (the size the closure
    is timed at; 256 tiles of the apply kernel) equals the FP64 reference on
    every cell."""
    from paper_1612_01287_gb300 import MLP, Sod, closure_step
    Z, tau = 65536, 0.05
    dt = 0.5 * (2.0 / Z)
    n, T0, b = workloads.random_smooth_fields(Z, beta_max=0.5)
    # a few sharp steps so that the difference features are not all small
    zc = (np.arange(Z) + 0.5) / Z
    n = n * np.where((zc > 0.3) & (zc < 0.3004), 0.5, 1.0)
    kw = dict(Z=Z, Q_xi=QLO, Q_L=QL, N_Omega=5, precision="f32", bc="outflow", tau=tau, dt=dt,
              fields=(n, T0, b))
    rng = np.random.default_rng(13)
    norm = random_norm(rng)
    with MLP(D, H, O, seed=6) as m, Sod(**kw) as a, Sod(**kw) as c:
        th = m.get_params()
        th[D * H + H + H * H + H:] *= 10.0
        m.set_params(th)
        m.set_normalization(*norm)
        a.step(1)
        closure_step(c, m, tau, 1)
        fa = a.get_state().astype(np.float64).T
        fc = c.get_state().astype(np.float64).T
        thr = oracle_theta(m.get_params())
    ref = C.correction(thr, fa, tau, QLO, QL, H, f64(norm))
    assert np.abs(ref).max() > 1e-4 * np.abs(fa).max()
    err = np.abs((fc - fa) - ref).max(axis=1)
    assert err.max() <= 1e-5 * np.abs(fa).max(), int(err.argmax())


def test_trained_closure_lowers_low_order_error():
    """Train on data the high-order method generates (Q_xi = 200; 24 tubes with
    tau log-uniform in [5e-3, 10] (dt = 2e-3 here; tau must exceed it), 12
    snapshots each, targets scaled per tau), then run
    Q_xi = 8 with and without the closure from the shock-tube state and compare
    the L2 errors of e and beta against Q_xi = 200: no tau is made worse (where
    the network explains less than 0.8 of the one-step target the plain
    low-order method runs), and the kinetic ones are improved."""
    from paper_1612_01287_gb300 import Sod
    from paper_1612_01287_gb300 import closure_train as CT
    Z, t_end = 512, 0.2
    dz = 2.0 / Z
    dt = 0.5 * dz / 0.9999
    nsteps = int(round(t_end / dt))
    rng = np.random.default_rng(workloads.SEED)
    taus = 10.0 ** rng.uniform(np.log10(5e-3), 1.0, size=24)
    steps = [sorted(rng.integers(0, nsteps, size=12).tolist()) for _ in taus]
    X, T, snaps = CT.generate(Z, taus, steps, dt)
    cl_model, losses = CT.train(X, T, snaps, epochs=30, batch=2048, lr=2e-3, seed=11)
    print("training samples", X.shape[0], "loss first/last epoch", losses[0], losses[-1])
    print("explained fraction by log10 tau:", np.round(cl_model.explained, 3).tolist())
    assert losses[-1] < 0.5 * losses[0]

    def l2(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    res = {}
    judged = (0.01, 0.1, 0.5, 1.0)
    with cl_model:
        for tau in judged:
            kw = dict(Z=Z, Q_L=QL, N_Omega=5, precision="f32", bc="outflow", tau=tau, dt=dt)
            with Sod(Q_xi=QHI, **kw) as hi, Sod(Q_xi=QLO, **kw) as lo, Sod(Q_xi=QLO, **kw) as cl:
                hi.step(nsteps)
                lo.step(nsteps)
                cl_model.step(cl, tau, nsteps)
                mh, ml, mc = hi.moments(), lo.moments(), cl.moments()
            res[tau] = {"plain": (l2(ml["E"], mh["E"]), l2(ml["beta"], mh["beta"])),
                        "closure": (l2(mc["E"], mh["E"]), l2(mc["beta"], mh["beta"]))}
    print("L2 errors (e, beta) vs Q_xi = 200:", res)
    for t in judged:
        assert res[t]["closure"][0] <= 1.05 * res[t]["plain"][0], (t, res)
    better = [res[t]["closure"][0] < res[t]["plain"][0] for t in judged if t >= 0.1]
    assert sum(better) >= 2, res
