"""Training data, training and use of the learned closure (an addition to the
paper's method; see rslb.h, "Learned closure").

Samples come from the method itself: for each relaxation time tau a
high-order tube (Q_xi = q_hi) and a low-order tube (Q_xi = q_lo) start from the
Sod state; the high-order tube is advanced to a sample time and
rslb_closure_sample restricts it to the low-order set and records the
features and the one-step target of every cell.

The targets shrink by orders of magnitude towards small tau (the low-order set
is already accurate near equilibrium), so a plain mean-squared loss would be
decided by the large-tau samples.  Each snapshot's targets are therefore
divided by a scale s(tau), interpolated log-log from the root-mean-square
targets of the snapshots, and the network learns the scaled targets: every tau
range weighs the same in the loss.  When the closure is applied at a given tau,
the network's output scale is multiplied by s(tau) for that call.

After training, the part of each snapshot's scaled one-step target that the
network reproduces, 1 - |T - net(X)|^2 / |T|^2, is binned in log tau like the
scale.  Where that explained fraction is below a gate (0.8), the network does
not know the one-step correction well enough at that tau and the low-order
method runs without it: the plain method is the fallback.  The residual of
every step adds up over a run; a network that explained 0.6 of the one-step
target at tau = 0.01 doubled the error of the plain low-order run there.
"""
import math

import numpy as np

QL_DEFAULT, Q_HI, Q_LO = 3, 200, 8


def _sod(Z, Q_xi, tau, dt, Q_L, stream):
    from . import Sod
    return Sod(Z=Z, Q_xi=Q_xi, Q_L=Q_L, N_Omega=5, precision="f32", bc="outflow", tau=tau,
               dt=dt, stream=stream)


def generate(Z, taus, sample_steps, dt, q_hi=Q_HI, q_lo=Q_LO, Q_L=QL_DEFAULT, stream=None):
    """Snapshots of (features, targets): for every tau, the high-order tube is
    advanced to each step count in sample_steps[i] (ascending) and sampled there.
    Returns X [N][3V+1], T [N][V] (torch float32 on the current device) and, per
    snapshot, (tau, first row, row count, rms of its targets)."""
    import torch
    from . import closure_sample
    V = Q_L * q_lo
    D = 3 * V + 1
    Xs, Ts, snaps, row = [], [], [], 0
    for tau, steps in zip(taus, sample_steps):
        with _sod(Z, q_hi, tau, dt, Q_L, stream) as hi, _sod(Z, q_lo, tau, dt, Q_L, stream) as lo:
            done = 0
            for n in steps:
                if n > done:
                    hi.step(n - done)
                    done = n
                X = torch.empty((Z, D), device="cuda")
                T = torch.empty((Z, V), device="cuda")
                closure_sample(hi, lo, tau, X.data_ptr(), T.data_ptr())
                done += 1  # the sample advanced both tubes one RK3 step
                rms = float(torch.sqrt(torch.mean(T.double() ** 2)).item())
                Xs.append(X)
                Ts.append(T)
                snaps.append((float(tau), row, Z, rms))
                row += Z
    return torch.cat(Xs).contiguous(), torch.cat(Ts).contiguous(), snaps


def scale_table(snaps, nodes=12):
    """(log10 tau nodes, log s) of the target scale: the log of the snapshot rms
    averaged in equal-width log-tau bins (empty bins skipped)."""
    lt = np.array([math.log10(s[0]) for s in snaps])
    lr = np.array([math.log(max(s[3], 1e-30)) for s in snaps])
    edges = np.linspace(lt.min(), lt.max() + 1e-12, nodes + 1)
    xs, ys = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        m = (lt >= a) & (lt < b)
        if m.any():
            xs.append(float(lt[m].mean()))
            ys.append(float(lr[m].mean()))
    return np.array(xs), np.array(ys)


def scale_at(tau, table):
    xs, ys = table
    return float(math.exp(np.interp(math.log10(tau), xs, ys)))


def explained_table(T, Y, snaps, nodes=12):
    """(log10 tau nodes, explained fraction): 1 - |T - Y|^2/|T|^2 of each
    snapshot's rows, averaged in the log-tau bins of scale_table."""
    lt = np.array([math.log10(s[0]) for s in snaps])
    ex = []
    for _, r0, n, _ in snaps:
        t, y = T[r0:r0 + n].double(), Y[r0:r0 + n].double()
        den = float((t * t).sum().item())
        ex.append(1.0 - float(((t - y) ** 2).sum().item()) / den if den > 0 else 0.0)
    ex = np.array(ex)
    edges = np.linspace(lt.min(), lt.max() + 1e-12, nodes + 1)
    xs, ys = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        m = (lt >= a) & (lt < b)
        if m.any():
            xs.append(float(lt[m].mean()))
            ys.append(float(ex[m].mean()))
    return np.array(xs), np.array(ys)


class Closure:
    """A trained network, its target scale table and its explained-fraction
    table; step() applies it where the explained fraction reaches the gate
    and runs the plain low-order method elsewhere."""

    def __init__(self, mlp, table, explained=None, gate=0.8):
        self.mlp = mlp
        self.table = table
        self.explained = explained
        self.gate = gate

    def active(self, tau):
        if self.explained is None:
            return True
        xs, ys = self.explained
        return float(np.interp(math.log10(tau), xs, ys)) >= self.gate

    def step(self, lo, tau, nsteps):
        from . import closure_step
        if not self.active(tau):
            lo.step(nsteps)
            return
        mu, isd, osd = self.mlp.get_normalization()
        self.mlp.set_normalization(mu, isd, osd * np.float32(scale_at(tau, self.table)))
        try:
            closure_step(lo, self.mlp, tau, nsteps)
        finally:
            self.mlp.set_normalization(mu, isd, osd)

    def close(self):
        self.mlp.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def train(X, T, snaps, hidden=64, epochs=40, batch=8192, lr=2e-3, seed=20161201, stream=None,
          nodes=12, max_z=20.0):
    """Scale each snapshot's targets by 1/s(tau) (in place), fit the fixed input
    and output normalisation (input scales widened so that no training input
    exceeds max_z in normalised units), train with Adam; returns (Closure,
    epoch losses); the Closure carries the explained-fraction table."""
    import torch
    from . import MLP
    table = scale_table(snaps, nodes)
    for tau, r0, n, _ in snaps:
        T[r0:r0 + n].mul_(1.0 / scale_at(tau, table))
    D, V = X.shape[1], T.shape[1]
    m = MLP(D, hidden, V, seed=seed, stream=stream)
    m.fit_normalization(X.data_ptr(), T.data_ptr(), X.shape[0])
    # most cells are smooth, so the fitted input deviations are small and the
    # cells at a discontinuity would reach hundreds of them: widen each
    # column's scale so that no training input lies beyond max_z of it
    mu, isd, osd = m.get_normalization()
    amax = (X - X.new_tensor(mu)).abs().amax(0).cpu().numpy()
    isd = np.minimum(isd, max_z / np.maximum(amax, 1e-30)).astype(np.float32)
    m.set_normalization(mu, isd, osd)
    losses = m.train(X.data_ptr(), T.data_ptr(), X.shape[0], epochs=epochs, batch=batch, lr=lr,
                     seed=seed + 1)
    Y = torch.empty_like(T)
    m.forward(X.data_ptr(), X.shape[0], Y.data_ptr())
    torch.cuda.synchronize()
    explained = explained_table(T, Y, snaps, nodes)
    del Y
    return Closure(m, table, explained), losses
