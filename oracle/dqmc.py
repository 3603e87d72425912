"""Plain DQMC Markov chain (test infrastructure; see package header).

One sweep = an up pass over slices l = 1..M followed by a down pass l = M..1
(the paper gives no sweep definition; this is the reading used on both sides):

  up,   l = 1..M:  G <- B_l G B_l^{-1}            (wrap tau_{l-1} -> tau_l)
                   propose every site i = 0..N-1 of slice l in index order
                   if l is a checkpoint: refresh G from the UDV stacks
  down, l = M..1:  propose every site of slice l in index order
                   G <- B_l^{-1} G B_l            (unwrap tau_l -> tau_{l-1})
                   if l-1 is a checkpoint: refresh G from the UDV stacks

Checkpoints tau_c = min(c * n_stab, M), c = 0..C, C = ceil(M / n_stab).
Stacks: right[c] = B(tau_c, 0) (built on the up pass), left[c] = B(beta, tau_c)
(built on the down pass, and once from the top at start-up); both are UDV
products with a column-pivoted QR after every slice (see ``green``).

Proposal for site i of slice l, with s = s_{il}:
  delta = e^{-2 lambda s} - 1,   r = 1 + delta (1 - G_ii),   R = e^{2 lambda s} r^2,
  accept iff u < R (u from Philox, one draw per proposal; ties rejected).
Accepting flips s and applies the Sherman-Morrison rank-one update
  G <- G - (delta / r) G[:, i] (e_i - G[i, :])^T.
The paper cites delayed updates for this step; grouping k such updates into
one rank-k product changes neither G nor any ratio in exact arithmetic, so the
oracle applies them one at a time.
"""

import math
import time

import numpy as np

from . import green, measure, philox
from .model import Model


class NumericError(RuntimeError):
    pass


class Chain:
    def __init__(self, L, beta, dtau, U, mu, seed, n_stab=10, chain=0, t=1.0, L2=None,
                 field=None, site_offsets=True, lattice="kagome"):
        self.model = Model(L, beta, dtau, U, mu, t=t, L2=L2, lattice=lattice)
        m = self.model
        self.N, self.M = m.N, m.M
        self.seed, self.chain = int(seed), int(chain)
        self.n_stab = int(n_stab)
        if self.n_stab < 1:
            raise ValueError("n_stab >= 1")
        C = -(-self.M // self.n_stab)
        self.tau = [min(c * self.n_stab, self.M) for c in range(C + 1)]
        self.C = C
        self.field = (philox.initial_field(seed, chain, self.M, self.N) if field is None
                      else np.array(field, dtype=np.int8).reshape(self.M, self.N).copy())
        self.sweeps_done = 0
        self.obs = measure.Observables(m.L1, m.L2, m.K, site_offsets, lattice_name=lattice)
        self.samples = []          # one dict per measurement
        self.max_drift = 0.0
        self.accepted = 0
        self.proposed = 0
        self._e2ls = {1: math.exp(2 * m.lam), -1: math.exp(-2 * m.lam)}
        self._delta = {1: math.exp(-2 * m.lam) - 1.0, -1: math.exp(2 * m.lam) - 1.0}
        self.reset_green()

    # --- stacks ---------------------------------------------------------------
    def _chunk_right(self, u, c):
        """right[c] = B_{tau_c} ... B_{tau_{c-1}+1} right[c-1]."""
        for l in range(self.tau[c - 1] + 1, self.tau[c] + 1):
            u.left_multiply(self.model.B(self.field[l - 1]))
        return u

    def _chunk_left(self, u, c):
        """left[c] = left[c+1] B_{tau_{c+1}} ... B_{tau_c+1}, kept transposed."""
        for l in range(self.tau[c + 1], self.tau[c], -1):
            u.left_multiply(self.model.BT(self.field[l - 1]))
        return u

    def reset_green(self):
        """Rebuild both stacks from the current field and set G = G(tau_0)."""
        self.left = [None] * (self.C + 1)
        self.right = [None] * (self.C + 1)
        self.left[self.C] = green.UDV(self.N)
        for c in range(self.C - 1, -1, -1):
            self.left[c] = self._chunk_left(self.left[c + 1].copy(), c)
        self.right[0] = green.UDV(self.N)
        self.G = green.combine(self.right[0], self.left[0])
        self.slice = 0

    # --- one slice of proposals -------------------------------------------------
    def update_slice(self, l, pas, forced=None):
        """Propose every site of slice l (1-based). ``forced`` (optional, bool per
        site) replaces the Metropolis decision: flip iff forced[i]."""
        m = self.model
        G = self.G
        N = self.N
        u = philox.metropolis_uniforms(self.seed, self.chain, self.sweeps_done, pas, l, N)
        s = self.field[l - 1]
        for i in range(N):
            si = int(s[i])
            delta = self._delta[si]
            r = 1.0 + delta * (1.0 - G[i, i])
            R = self._e2ls[si] * r * r
            if not (R > 0.0) or not math.isfinite(R):
                raise NumericError(f"non-positive or non-finite ratio {R} at slice {l} site {i}")
            self.proposed += 1
            acc = bool(forced[i]) if forced is not None else (u[i] < R)
            if acc:
                self.accepted += 1
                col = G[:, i].copy()
                row = -G[i, :].copy()
                row[i] += 1.0
                G -= (delta / r) * np.outer(col, row)
                s[i] = -si
        self.G = G

    def _refresh(self, c):
        G_fresh = green.combine(self.right[c], self.left[c])
        self.max_drift = max(self.max_drift, float(np.max(np.abs(G_fresh - self.G))))
        self.G = G_fresh

    def sweep(self, measure_obs=False, forced=None):
        """One up + down sweep. ``forced``: optional (2, M, N) bool array of
        imposed decisions (pass, slice-1, site) for replays."""
        m = self.model
        c = 1
        for l in range(1, self.M + 1):
            self.G = m.B(self.field[l - 1]) @ self.G @ m.Binv(self.field[l - 1])
            self.update_slice(l, 0, None if forced is None else forced[0, l - 1])
            self.slice = l
            if l == self.tau[c]:
                self.right[c] = self._chunk_right(self.right[c - 1].copy(), c)
                self._refresh(c)
                if measure_obs and self._measure_at(c):
                    self.samples.append(self.obs(self.G))
                c += 1
        c = self.C - 1
        for l in range(self.M, 0, -1):
            self.update_slice(l, 1, None if forced is None else forced[1, l - 1])
            self.G = m.Binv(self.field[l - 1]) @ self.G @ m.B(self.field[l - 1])
            self.slice = l - 1
            if l - 1 == self.tau[c]:
                self.left[c] = self._chunk_left(self.left[c + 1].copy(), c)
                self._refresh(c)
                c -= 1
        self.sweeps_done += 1

    def _measure_at(self, c):
        """Up-pass checkpoints at which measurements are taken: all of them."""
        return True

    def run(self, n_sweeps, measure_obs=False):
        for _ in range(n_sweeps):
            self.sweep(measure_obs)

    # --- helpers for parity tests -------------------------------------------------
    def green_fresh(self, l):
        """From-scratch stabilised G(tau_l) for the current field."""
        return green.green_udv(self.model, self.field, l)

    def bins(self, bin_size):
        keys = measure.Observables.NAMES
        x = np.array([[smp[k] for k in keys] for smp in self.samples])
        nb = len(x) // bin_size
        return x[:nb * bin_size].reshape(nb, bin_size, len(keys)).mean(axis=1)


def time_slice_visits(L, beta, dtau, U, mu, seed, n_visits, n_stab=8, with_refresh=True):
    """Wall time of ``n_visits`` up-pass slice visits (wrap + N proposals, and
    with_refresh: the stack update and refresh at checkpoints) after start-up;
    returns (seconds, proposals, number of refreshes). Used for the CPU
    baseline. Without refresh the chain starts from the U = 0 closed-form G
    (no start-up stack build, which at L = 24 alone takes minutes)."""
    ch = Chain.__new__(Chain)
    ch.model = Model(L, beta, dtau, U, mu)
    m = ch.model
    ch.N, ch.M, ch.seed, ch.chain, ch.n_stab = m.N, m.M, int(seed), 0, int(n_stab)
    ch.C = -(-ch.M // ch.n_stab)
    ch.tau = [min(c * ch.n_stab, ch.M) for c in range(ch.C + 1)]
    ch.field = philox.initial_field(seed, 0, ch.M, ch.N)
    ch.sweeps_done, ch.max_drift, ch.accepted, ch.proposed = 0, 0.0, 0, 0
    ch._e2ls = {1: math.exp(2 * m.lam), -1: math.exp(-2 * m.lam)}
    ch._delta = {1: math.exp(-2 * m.lam) - 1.0, -1: math.exp(2 * m.lam) - 1.0}
    if with_refresh:
        ch.reset_green()
    else:
        ch.G = m.green_free()
    t0 = time.perf_counter()
    c = 1
    refreshes = 0
    for l in range(1, n_visits + 1):
        ch.G = m.B(ch.field[l - 1]) @ ch.G @ m.Binv(ch.field[l - 1])
        ch.update_slice(l, 0)
        if with_refresh and l == ch.tau[c]:
            ch.right[c] = ch._chunk_right(ch.right[c - 1].copy(), c)
            ch._refresh(c)
            refreshes += 1
            c += 1
    return time.perf_counter() - t0, n_visits * ch.N, refreshes
