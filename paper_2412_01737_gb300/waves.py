"""Residency waves: more chains than fit in HBM on one GPU.

A context holds the inverses of one wave of chains on the device; the other
waves' states live in host memory (on a Grace-Hopper/Blackwell superchip the
CPU's memory, reached over NVLink-C2C) and are swapped in with
``GGF.load_state`` and out with ``GGF.save_state``.  A swap copies the chains'
exact state, so every wave continues bit for bit as if it had stayed
resident; no inverse is refactorised.  Wave w's chains use the Philox key
(seed + 7919 w, chain), so the waves' random streams are distinct.
"""
from __future__ import annotations

import numpy as np


class Waves:
    """n_waves waves of the context's chain count, states held on the host."""

    def __init__(self, ctx, start_links: list, seed: int, pinned: bool = True, **chain_opts):
        """start_links[w]: the wave's starting links (all waves the same shape);
        chain_opts: the remaining GGF.chains_init options."""
        self.ctx = ctx
        self.seeds = [seed + 7919 * w for w in range(len(start_links))]
        self.states = []
        for w, links in enumerate(start_links):
            ctx.chains_init(links, seed=self.seeds[w], **chain_opts)
            buf = self._buffer(ctx.state_size(), pinned)
            ctx.save_state(buf)
            self.states.append(buf)

    @staticmethod
    def _buffer(nbytes: int, pinned: bool):
        if pinned:
            try:
                import torch
                if torch.cuda.is_available():
                    return torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
            except ImportError:
                pass
        return np.empty(nbytes, dtype=np.uint8)

    def sample(self, n_sweeps: int):
        """n_sweeps sweeps of every wave in turn; returns the observables
        [n_waves, n_sweeps, chains, 3]."""
        out = []
        for buf in self.states:
            self.ctx.load_state(buf)
            out.append(self.ctx.sample(n_sweeps))
            self.ctx.save_state(buf)
        return np.array(out)

    def links(self):
        """Current links of every wave, [n_waves, chains, ...]."""
        out = []
        for buf in self.states:
            self.ctx.load_state(buf)
            out.append(self.ctx.chains_links())
        return np.array(out)
