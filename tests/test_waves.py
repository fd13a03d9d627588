"""Host logic of the residency-wave driver (paper_2412_01737_gb300/waves.py)
with a stand-in context whose whole state is a small array: every wave is
initialised with its own seed, saved, and sampled in turn from its own
state, and its history equals that of a context that never swapped."""
import numpy as np

from paper_2412_01737_gb300.waves import Waves


class _Ctx:
    """Chains whose state is (seed, sweep, links); a sweep adds seed + sweep."""

    def chains_init(self, links, seed=0, **opts):
        self.state = np.concatenate([[seed, 0], np.asarray(links, dtype=np.float64).ravel()])
        self.shape = np.asarray(links).shape

    def state_size(self):
        return self.state.nbytes

    def save_state(self, out=None):
        out = np.empty(self.state_size(), dtype=np.uint8) if out is None else out
        out[:] = self.state.view(np.uint8)
        return out

    def load_state(self, src):
        self.state = np.asarray(src).view(np.float64).copy()

    def sample(self, n):
        obs = []
        for _ in range(n):
            self.state[2:] += self.state[0] + self.state[1]
            self.state[1] += 1
            obs.append(self.state[2:].reshape(self.shape)[:, :1].repeat(3, axis=1))
        return np.array(obs)

    def chains_links(self):
        return self.state[2:].reshape(self.shape).copy()


def test_waves_reproduce_resident_chains():
    starts = [np.arange(6.0).reshape(3, 2), 10 + np.arange(6.0).reshape(3, 2)]
    wv = Waves(_Ctx(), starts, seed=5, pinned=False, precision=0)
    o1, o2, links = wv.sample(2), wv.sample(3), wv.links()
    for w in range(2):
        c = _Ctx()
        c.chains_init(starts[w], seed=5 + 7919 * w)
        assert np.array_equal(o1[w], c.sample(2))
        assert np.array_equal(o2[w], c.sample(3))
        assert np.array_equal(links[w], c.chains_links())
