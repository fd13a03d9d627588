"""ctypes binding of libggf (include/ggf.h).  Argument marshalling only.

Arrays may be numpy arrays (host memory: the library copies in and out) or
torch CUDA tensors (device memory, borrowed for the call on torch's current
stream).  Every entry point of the C ABI has a method of the same name here
(without the ggf_ prefix).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

Z2, U1, SU2 = 0, 1, 2
PAIRS_NORM, PAIRS_ELECTRIC, PAIRS_SITE, PAIRS_LINK, PAIRS_FIELD, PAIRS_FOUR = 0, 1, 2, 3, 4, 5
FP64, FP32 = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
N_OBS = 3
OBS_PLAQUETTE = 0
KT_RATIO, KT_UPDATE, KT_REFRESH, KT_FLUSH, KT_GATHER, KT_APPLY = 0, 1, 2, 3, 4, 5

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libggf.so")
_lib = None

GGF_OK, GGF_ESINGULAR, GGF_EDRIFT = 0, 4, 6
STATUS = {0: "GGF_OK", 1: "GGF_EINVAL", 2: "GGF_ENOMEM", 3: "GGF_ECUDA", 4: "GGF_ESINGULAR",
          5: "GGF_ETIMEOUT", 6: "GGF_EDRIFT", 7: "GGF_ESTATE", 8: "GGF_EIO"}


class GGFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class ChainOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("refresh_every", ctypes.c_int), ("width", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("delay", ctypes.c_int), ("graph", ctypes.c_int),
                ("chain_offset", ctypes.c_uint64)]


class ChainStats(ctypes.Structure):
    _fields_ = [("proposals", ctypes.c_uint64), ("accepts", ctypes.c_uint64), ("refreshes", ctypes.c_uint64),
                ("sweeps", ctypes.c_uint64), ("max_drift", ctypes.c_double), ("launches", ctypes.c_uint64),
                ("block_proposals", ctypes.c_uint64), ("block_accepts", ctypes.c_uint64),
                ("n_chains", ctypes.c_int), ("n_pairs", ctypes.c_int), ("max_resid", ctypes.c_double),
                ("dense_refreshes", ctypes.c_uint64), ("refine_steps", ctypes.c_uint64),
                ("dense_pfaffians", ctypes.c_uint64), ("flush_wave", ctypes.c_uint64)]


EXPORTS = ["ggf_create", "ggf_destroy", "ggf_last_error", "ggf_init_lattice", "ggf_init_group",
           "ggf_init_gaussians", "ggf_get_constants", "ggf_logweight", "ggf_observable", "ggf_chains_init",
           "ggf_sample", "ggf_sample_group", "ggf_chains_links", "ggf_chains_ell", "ggf_chains_inverse",
           "ggf_chains_electric", "ggf_chains_fermion", "ggf_chains_pairs", "ggf_chains_score",
           "ggf_chains_fermion4", "ggf_chains_link_score", "ggf_wilson_loop", "ggf_polyakov_loop",
           "ggf_debug_poison_inverse", "ggf_chains_refine", "ggf_debug_scale_inverse", "ggf_chains_status", "ggf_chains_state_size", "ggf_chains_save_state", "ggf_chains_load_state",
           "ggf_chains_electric_field", "ggf_chains_link_terms",
           "ggf_chains_stats",
           "ggf_checkpoint",
           "ggf_resume", "ggf_profile", "ggf_kernel_time", "ggf_sync", "ggf_logweight_noalloc",
           "ggf_selftest_flush", "ggf_selftest_flush_data", "ggf_net_create", "ggf_net_destroy", "ggf_net_last_error", "ggf_net_get_params",
           "ggf_net_set_params", "ggf_net_logq", "ggf_net_loss_grad", "ggf_net_train", "ggf_sample_blocks"]


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libggf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libggf.so not built at {_LIB_PATH}; run paper_2412_01737_gb300.build.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    sig = {
        "ggf_create": ([ctypes.POINTER(P), I], I),
        "ggf_destroy": ([P], V),
        "ggf_last_error": ([P], ctypes.c_char_p),
        "ggf_init_lattice": ([P, I], I),
        "ggf_init_group": ([P, I, I, P], I),
        "ggf_init_gaussians": ([P, P, I, P, P], I),
        "ggf_get_constants": ([P, ctypes.POINTER(I), P, P], I),
        "ggf_logweight": ([P, I, P, P, P, I, P], I),
        "ggf_observable": ([P, I, I, P, P, I, P], I),
        "ggf_chains_init": ([P, I, P, ctypes.POINTER(ChainOpts), I, P], I),
        "ggf_sample": ([P, I, P, I, P], I),
        "ggf_sample_group": ([P, I, I, P, I, P], I),
        "ggf_chains_links": ([P, P, I, P], I),
        "ggf_chains_ell": ([P, P, I, P], I),
        "ggf_chains_inverse": ([P, I, I, P, I, P], I),
        "ggf_chains_electric": ([P, P, I, P], I),
        "ggf_chains_fermion": ([P, P, P, I, P], I),
        "ggf_chains_pairs": ([P, I, P, I, P], I),
        "ggf_chains_score": ([P, P, I, P], I),
        "ggf_chains_fermion4": ([P, P, I, P], I),
        "ggf_chains_link_score": ([P, P, I, P], I),
        "ggf_wilson_loop": ([P, I, I, I, P, P, I, P], I),
        "ggf_polyakov_loop": ([P, I, P, P, I, P], I),
        "ggf_debug_poison_inverse": ([P, I, I, I, I], I),
        "ggf_chains_refine": ([P, I, I, I, ctypes.POINTER(ctypes.c_double)], I),
        "ggf_debug_scale_inverse": ([P, I, I, ctypes.c_double], I),
        "ggf_chains_status": ([P, ctypes.c_double, P, I, P], I),
        "ggf_chains_electric_field": ([P, P, I, P], I),
        "ggf_chains_link_terms": ([P, P, P, P, I, P], I),
        "ggf_chains_state_size": ([P, ctypes.POINTER(ctypes.c_uint64)], I),
        "ggf_chains_save_state": ([P, P, I, P], I),
        "ggf_chains_load_state": ([P, P, I, P], I),
        "ggf_chains_stats": ([P, ctypes.POINTER(ChainStats)], I),
        "ggf_checkpoint": ([P, ctypes.c_char_p], I),
        "ggf_resume": ([P, ctypes.c_char_p, P], I),
        "ggf_profile": ([P, I], I),
        "ggf_kernel_time": ([P, I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)], I),
        "ggf_sync": ([P, P], I),
        "ggf_logweight_noalloc": ([P, I, P, P, P], I),
        "ggf_selftest_flush": ([P, I, I, I, ctypes.POINTER(ctypes.c_double)], I),
        "ggf_selftest_flush_data": ([P, I, I, I, I, P, P, P], I),
        "ggf_net_create": ([ctypes.POINTER(P), I, I, ctypes.c_uint64], I),
        "ggf_net_destroy": ([P], V),
        "ggf_net_last_error": ([P], ctypes.c_char_p),
        "ggf_net_get_params": ([P, P], I),
        "ggf_net_set_params": ([P, P], I),
        "ggf_net_logq": ([P, I, P, P, P, I, P], I),
        "ggf_net_loss_grad": ([P, I, P, P, ctypes.POINTER(ctypes.c_double), P], I),
        "ggf_net_train": ([P, I, P, I, I, ctypes.c_float, P, P], I),
        "ggf_sample_blocks": ([P, P, I, P, I, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(a):
    """(pointer, mem) of a numpy array or torch CUDA tensor."""
    if a is None:
        return None, MEM_HOST
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous (use np.ascontiguousarray)")
        return a.ctypes.data, MEM_HOST
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), (MEM_DEVICE if a.is_cuda else MEM_HOST)
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(arrs):
    for a in arrs:
        if a is not None and hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


class GGF:
    """One libggf context on a CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.ggf_create(ctypes.byref(h), device)
        if st != 0:
            raise GGFError(st, "ggf_create failed (no CUDA device?)")
        self.h = h
        self.group = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.ggf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        if st != 0:
            raise GGFError(st, self.lib.ggf_last_error(self.h).decode())

    def _mem(self, *arrs):
        mems = {_ptr(a)[1] for a in arrs if a is not None}
        if len(mems) > 1:
            raise ValueError("mix of host and device arrays in one call")
        return mems.pop() if mems else MEM_HOST

    # ---- set-up -------------------------------------------------------------
    def init_lattice(self, L):
        self._ck(self.lib.ggf_init_lattice(self.h, int(L)))
        self._n_links = 2 * int(L) * int(L)

    def init_group(self, group, n_v, q_src=None):
        self.group = int(group)
        self.n_v = int(n_v)
        q = None if q_src is None else np.ascontiguousarray(q_src, dtype=np.int32)
        self._ck(self.lib.ggf_init_group(self.h, int(group), int(n_v), None if q is None else q.ctypes.data))

    def init_gaussians(self, gamma_site, K, gamma_bond, lam):
        gs = np.ascontiguousarray(gamma_site, dtype=np.float64)
        gb = np.ascontiguousarray(gamma_bond, dtype=np.float64)
        lm = np.ascontiguousarray(np.stack([np.real(lam), np.imag(lam)], axis=-1), dtype=np.float64)
        self._ck(self.lib.ggf_init_gaussians(self.h, gs.ctypes.data, int(K), gb.ctypes.data, lm.ctypes.data))
        self.K = int(K)

    def init_problem(self, p):
        """Convenience: the three init calls for a ggf_inputs.Problem-like object."""
        self.init_lattice(p.L)
        self.init_group(p.group, p.n_v, p.q_src)
        self.init_gaussians(p.gamma_site, p.K, p.gamma_bond, p.lam)

    def get_constants(self):
        n = ctypes.c_int()
        self._ck(self.lib.ggf_get_constants(self.h, ctypes.byref(n), None, None))
        lc = np.zeros((n.value, 2))
        pr = np.zeros((n.value, 2), dtype=np.int32)
        self._ck(self.lib.ggf_get_constants(self.h, ctypes.byref(n), lc.ctypes.data, pr.ctypes.data))
        return lc[:, 0] + 1j * lc[:, 1], pr

    # ---- compute --------------------------------------------------------------
    def logweight(self, links, logN=None, ell=None):
        """log N(G) per configuration (and log Pf(M_nm) per pair into `ell`)."""
        n_cfg = int(links.shape[0])
        if logN is None:
            logN = np.zeros(n_cfg) if isinstance(links, np.ndarray) else _torch_like(links, (n_cfg,))
        mem = self._mem(links, logN, ell)
        lp, _ = _ptr(links)
        self._ck(self.lib.ggf_logweight(self.h, n_cfg, lp, _ptr(logN)[0], _ptr(ell)[0], mem,
                                        _stream([links, logN, ell])))
        return logN

    def logweight_noalloc(self, links, logN, stream=None):
        """Allocation-free log N(G) into `logN`; both are CUDA tensors."""
        if _ptr(links)[1] != MEM_DEVICE or _ptr(logN)[1] != MEM_DEVICE:
            raise ValueError("logweight_noalloc takes device tensors only")
        st = stream if stream is not None else _stream([links, logN])
        self._ck(self.lib.ggf_logweight_noalloc(self.h, int(links.shape[0]), _ptr(links)[0], _ptr(logN)[0], st))
        return logN

    def observable(self, links, out=None, which=OBS_PLAQUETTE):
        n_cfg = int(links.shape[0])
        if out is None:
            out = np.zeros(n_cfg) if isinstance(links, np.ndarray) else _torch_like(links, (n_cfg,))
        mem = self._mem(links, out)
        self._ck(self.lib.ggf_observable(self.h, which, n_cfg, _ptr(links)[0], _ptr(out)[0], mem,
                                         _stream([links, out])))
        return out

    def wilson_loop(self, links, R, T, out=None):
        """Mean R x T Wilson loop of every configuration (Sec. 5.1)."""
        n_cfg = int(links.shape[0])
        if out is None:
            out = np.zeros(n_cfg) if isinstance(links, np.ndarray) else _torch_like(links, (n_cfg,))
        self._ck(self.lib.ggf_wilson_loop(self.h, int(R), int(T), n_cfg, _ptr(links)[0], _ptr(out)[0],
                                          self._mem(links, out), _stream([links, out])))
        return out

    def polyakov_loop(self, links, out=None):
        """Mean loop winding along y of every configuration."""
        n_cfg = int(links.shape[0])
        if out is None:
            out = np.zeros(n_cfg) if isinstance(links, np.ndarray) else _torch_like(links, (n_cfg,))
        self._ck(self.lib.ggf_polyakov_loop(self.h, n_cfg, _ptr(links)[0], _ptr(out)[0], self._mem(links, out),
                                            _stream([links, out])))
        return out

    def chains_init(self, links, precision=FP64, refresh_every=64, width=0.5, seed=20241202, delay=1, graph=1,
                    chain_offset=0):
        o = ChainOpts(int(precision), int(refresh_every), float(width), int(seed), int(delay), int(graph),
                      int(chain_offset))
        mem = self._mem(links)
        self.n_chains = int(links.shape[0])
        self.link_dtype = links.dtype
        self._ck(self.lib.ggf_chains_init(self.h, self.n_chains, _ptr(links)[0], ctypes.byref(o), mem,
                                          _stream([links])))

    def sample(self, n_sweeps, obs=None):
        """Run sweeps; returns obs [n_sweeps, n_chains, 3] (numpy unless a tensor is given)."""
        if obs is None:
            obs = np.zeros((int(n_sweeps), self.n_chains, N_OBS))
        mem = self._mem(obs)
        self._ck(self.lib.ggf_sample(self.h, int(n_sweeps), _ptr(obs)[0], mem, _stream([obs])))
        return obs

    def sample_no_obs(self, n_sweeps, stream=None):
        self._ck(self.lib.ggf_sample(self.h, int(n_sweeps), None, MEM_DEVICE, stream))

    def sample_blocks(self, net, n_moves, obs=None):
        """Learned-proposal block moves; returns obs [n_moves, n_chains, 3]."""
        if obs is None:
            obs = np.zeros((int(n_moves), self.n_chains, N_OBS))
        self._ck(self.lib.ggf_sample_blocks(self.h, net.h, int(n_moves), _ptr(obs)[0], self._mem(obs), _stream([obs])))
        return obs

    def chains_links(self, out=None):
        if out is None:
            L = self.n_links()
            if self.group == SU2:
                out = np.zeros((self.n_chains, L, 4))          # unit quaternions
            else:
                out = np.zeros((self.n_chains, L), dtype=np.int8 if self.group == Z2 else np.float64)
        self._ck(self.lib.ggf_chains_links(self.h, _ptr(out)[0], self._mem(out), _stream([out])))
        return out

    def chains_ell(self):
        st = self.chains_stats()
        out = np.zeros((self.n_chains, st.n_pairs, 2))
        self._ck(self.lib.ggf_chains_ell(self.h, out.ctypes.data, MEM_HOST, None))
        return out[..., 0] + 1j * out[..., 1]

    def chains_electric(self, out=None):
        """f_E(G)_l of every chain and link (Sec. 5.3; Z2: the link flip,
        U(1): the Casimir J^2): complex numpy array (n_chains, 2V), or fills
        `out` (float64 [n_chains][2V][2], numpy or CUDA tensor) and returns it."""
        if out is None:
            host = np.zeros((self.n_chains, self.n_links(), 2))
            self._ck(self.lib.ggf_chains_electric(self.h, host.ctypes.data, MEM_HOST, None))
            return host[..., 0] + 1j * host[..., 1]
        self._ck(self.lib.ggf_chains_electric(self.h, _ptr(out)[0], self._mem(out), _stream([out])))
        return out

    def chains_electric_field(self, out=None):
        """U(1) electric field <J_l> of every chain and link (Sec. 5.3):
        complex numpy array (n_chains, 2V), or fills `out` (float64 [n][2V][2])."""
        if out is None:
            host = np.zeros((self.n_chains, self.n_links(), 2))
            self._ck(self.lib.ggf_chains_electric_field(self.h, host.ctypes.data, MEM_HOST, None))
            return host[..., 0] + 1j * host[..., 1]
        self._ck(self.lib.ggf_chains_electric_field(self.h, _ptr(out)[0], self._mem(out), _stream([out])))
        return out

    def chains_link_terms(self, charges, out=None, pair_out=None, pairs=False):
        """Gauge-invariant link terms T_l = u_l <F_s F_t> of every chain and
        link (charges: the sites' physical charges, +1 / -1).  Returns a
        complex numpy array (n_chains, 2V), with pairs=True also the per-pair
        parts (n_chains, 2V, K, K); or fills out [n][2V][2] and/or pair_out
        [n][2V][K][K][2] (numpy or CUDA tensors) and returns them."""
        q = np.ascontiguousarray(np.asarray(charges), dtype=np.int32)
        if q.shape != (self.n_links() // 2,):
            raise ValueError("charges must have one entry per site")
        if out is None and pair_out is None:
            host = np.zeros((self.n_chains, self.n_links(), 2))
            hp = np.zeros((self.n_chains, self.n_links(), self.K, self.K, 2)) if pairs else None
            self._ck(self.lib.ggf_chains_link_terms(self.h, q.ctypes.data, host.ctypes.data,
                                                    None if hp is None else hp.ctypes.data, MEM_HOST, None))
            T = host[..., 0] + 1j * host[..., 1]
            return (T, hp[..., 0] + 1j * hp[..., 1]) if pairs else T
        mem = self._mem(out, pair_out)
        self._ck(self.lib.ggf_chains_link_terms(self.h, q.ctypes.data, None if out is None else _ptr(out)[0],
                                                None if pair_out is None else _ptr(pair_out)[0], mem,
                                                _stream([a for a in (out, pair_out) if a is not None])))
        return out, pair_out

    def chains_fermion(self, site=None, link=None):
        """Physical Majorana bilinears of every chain (Sec. 5.2): complex numpy
        arrays site (n_chains, V) and link (n_chains, 2V, 2, 2); or fills the
        given float64 buffers site [n][V][2] / link [n][2V][2][2][2] (numpy or
        CUDA tensors, either may be None) and returns them."""
        if site is None and link is None:
            nl = self.n_links()
            hs = np.zeros((self.n_chains, nl // 2, 2))
            hl = np.zeros((self.n_chains, nl, 2, 2, 2))
            self._ck(self.lib.ggf_chains_fermion(self.h, hs.ctypes.data, hl.ctypes.data, MEM_HOST, None))
            return hs[..., 0] + 1j * hs[..., 1], hl[..., 0] + 1j * hl[..., 1]
        self._ck(self.lib.ggf_chains_fermion(self.h, _ptr(site)[0], _ptr(link)[0], self._mem(site, link),
                                             _stream([site, link])))
        return site, link

    def chains_pairs(self, what, out=None):
        """Per-pair parts N_nm(G) o_nm(G) / N(G) of every chain (PAIRS_NORM,
        PAIRS_ELECTRIC, PAIRS_SITE, PAIRS_LINK, PAIRS_FIELD, PAIRS_FOUR): complex arrays of shape
        (n_chains, [items...,] K, K), or fills `out` (float64 with a trailing
        axis of 2, numpy or CUDA tensor) and returns it."""
        if out is None:
            K = self.K
            nl = self.n_links()
            items = {PAIRS_NORM: (), PAIRS_ELECTRIC: (nl,), PAIRS_SITE: (nl // 2,), PAIRS_LINK: (nl, 2, 2),
                     PAIRS_FIELD: (nl,), PAIRS_FOUR: (nl,)}.get(what, ())
            host = np.zeros((self.n_chains,) + items + (K, K, 2))
            self._ck(self.lib.ggf_chains_pairs(self.h, int(what), host.ctypes.data, MEM_HOST, None))
            return host[..., 0] + 1j * host[..., 1]
        self._ck(self.lib.ggf_chains_pairs(self.h, int(what), _ptr(out)[0], self._mem(out), _stream([out])))
        return out

    def chains_link_score(self, out=None):
        """Per-pair link-block scores (n_chains, P, 2V, r, r) complex (see
        ggf_chains_link_score), or fills `out` (float64 with a trailing 2)."""
        if out is None:
            P = self.K * (self.K + 1) // 2
            r = 4 * self.n_v
            host = np.zeros((self.n_chains, P, self.n_links(), r, r, 2))
            self._ck(self.lib.ggf_chains_link_score(self.h, host.ctypes.data, MEM_HOST, None))
            return host[..., 0] + 1j * host[..., 1]
        self._ck(self.lib.ggf_chains_link_score(self.h, _ptr(out)[0], self._mem(out), _stream([out])))
        return out

    def chains_fermion4(self, out=None):
        """<c_2s c_2s+1 c_2t c_2t+1> per chain and link (s -> t): complex numpy
        array (n_chains, 2V), or fills `out` (float64 [n][2V][2])."""
        if out is None:
            host = np.zeros((self.n_chains, self.n_links(), 2))
            self._ck(self.lib.ggf_chains_fermion4(self.h, host.ctypes.data, MEM_HOST, None))
            return host[..., 0] + 1j * host[..., 1]
        self._ck(self.lib.ggf_chains_fermion4(self.h, _ptr(out)[0], self._mem(out), _stream([out])))
        return out

    def chains_score(self, out=None):
        """d log N(G) / d D_s of every chain and site: numpy array
        (n_chains, V, B, B), or fills `out` (float64, numpy or CUDA tensor)."""
        if out is None:
            nv = self.n_v
            host = np.zeros((self.n_chains, self.n_links() // 2, 8 * nv, 8 * nv))
            self._ck(self.lib.ggf_chains_score(self.h, host.ctypes.data, MEM_HOST, None))
            return host
        self._ck(self.lib.ggf_chains_score(self.h, _ptr(out)[0], self._mem(out), _stream([out])))
        return out

    def chains_inverse(self, chain, pair, N):
        out = np.zeros((N, N, 2))
        self._ck(self.lib.ggf_chains_inverse(self.h, int(chain), int(pair), out.ctypes.data, MEM_HOST, None))
        return out[..., 0] + 1j * out[..., 1]

    def chains_refine(self, chain, pair, apply=True):
        """max |I - M W| of one FP32 chain's cached inverse; with apply, one
        Newton step on the tensor cores follows (skipped above 1e-3)."""
        r = ctypes.c_double()
        self._ck(self.lib.ggf_chains_refine(self.h, int(chain), int(pair), 1 if apply else 0, ctypes.byref(r)))
        return r.value

    def debug_scale_inverse(self, chain, pair, factor):
        """Test hook: multiply one FP32 chain's cached inverse by `factor`."""
        self._ck(self.lib.ggf_debug_scale_inverse(self.h, int(chain), int(pair), float(factor)))

    def debug_poison_inverse(self, chain, pair, i, j):
        """Fault injection for tests: NaN into W_pair[i][j] of one chain."""
        self._ck(self.lib.ggf_debug_poison_inverse(self.h, int(chain), int(pair), int(i), int(j)))

    def chains_status(self, drift_tol=0.0):
        """Per-chain status codes (GGF_OK, GGF_ESINGULAR, GGF_EDRIFT), int32 numpy array."""
        out = np.zeros(self.n_chains, dtype=np.int32)
        self._ck(self.lib.ggf_chains_status(self.h, float(drift_tol), out.ctypes.data, MEM_HOST, None))
        return out

    def chains_stats(self):
        s = ChainStats()
        self._ck(self.lib.ggf_chains_stats(self.h, ctypes.byref(s)))
        return s

    def state_size(self):
        """Bytes of the in-memory chain state (save_state / load_state)."""
        n = ctypes.c_uint64()
        self._ck(self.lib.ggf_chains_state_size(self.h, ctypes.byref(n)))
        return n.value

    def save_state(self, out=None):
        """Copy the chains' state into `out` (uint8 numpy array or CUDA/pinned
        torch tensor of state_size() bytes; a new numpy array if None)."""
        if out is None:
            out = np.zeros(self.state_size(), dtype=np.uint8)
        self._ck(self.lib.ggf_chains_save_state(self.h, _ptr(out)[0], self._mem(out), _stream([out])))
        return out

    def load_state(self, src):
        """Replace the chains' state by a saved one of the same problem and shape."""
        self._ck(self.lib.ggf_chains_load_state(self.h, _ptr(src)[0], self._mem(src), _stream([src])))

    def checkpoint(self, path):
        self._ck(self.lib.ggf_checkpoint(self.h, str(path).encode()))

    def resume(self, path):
        self._ck(self.lib.ggf_resume(self.h, str(path).encode(), None))
        self.n_chains = self.chains_stats().n_chains

    def selftest_flush(self, cplx, N, rank):
        """Max relative error of the tensor-core flush against FP64."""
        e = ctypes.c_double()
        self._ck(self.lib.ggf_selftest_flush(self.h, int(cplx), int(N), int(rank), ctypes.byref(e)))
        return e.value

    def selftest_flush_data(self, cplx, N, rank, which):
        """(w0, panels, w1) of the flush self-test case as host arrays (see
        ggf_selftest_flush_data for the layouts)."""
        NP = (N + 255) // 256 * 256
        KP = (rank + 7) // 8 * 8
        nW = N * N * (2 if cplx else 1)
        w0 = np.zeros(nW, dtype=np.float32)
        w1 = np.zeros(nW, dtype=np.float32)
        pan = np.zeros((4 if cplx else 2) * NP * KP, dtype=np.float32)
        self._ck(self.lib.ggf_selftest_flush_data(self.h, int(cplx), int(N), int(rank), int(which),
                                                  w0.ctypes.data, pan.ctypes.data, w1.ctypes.data))
        return w0, pan, w1

    def profile(self, enable=True):
        self._ck(self.lib.ggf_profile(self.h, 1 if enable else 0))

    def kernel_time(self, which):
        """(milliseconds, launches) accumulated since profile(True)."""
        ms, n = ctypes.c_double(), ctypes.c_uint64()
        self._ck(self.lib.ggf_kernel_time(self.h, int(which), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def sync(self, stream=None):
        self._ck(self.lib.ggf_sync(self.h, stream))

    def n_links(self):
        return getattr(self, "_n_links", None) or self._links_from_state()

    def _links_from_state(self):
        raise RuntimeError("call init_problem/init_lattice through this object first")


NET_PARAMS = 81990


class Net:
    """The learned block-proposal network (ggf_net)."""

    def __init__(self, device: int, L: int, seed: int = 1):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.ggf_net_create(ctypes.byref(h), int(device), int(L), int(seed))
        if st != 0:
            raise GGFError(st, "ggf_net_create failed")
        self.h, self.L = h, int(L)

    def close(self):
        if getattr(self, "h", None):
            self.lib.ggf_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        if st != 0:
            raise GGFError(st, self.lib.ggf_net_last_error(self.h).decode())

    def get_params(self):
        out = np.zeros(NET_PARAMS, dtype=np.float32)
        self._ck(self.lib.ggf_net_get_params(self.h, out.ctypes.data))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._ck(self.lib.ggf_net_set_params(self.h, p.ctypes.data))

    def logq(self, theta, blocks):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        bl = np.ascontiguousarray(blocks, dtype=np.int32)
        out = np.zeros(len(th))
        self._ck(self.lib.ggf_net_logq(self.h, len(th), th.ctypes.data, bl.ctypes.data, out.ctypes.data, MEM_HOST,
                                       None))
        return out

    def loss_grad(self, theta, blocks):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        bl = np.ascontiguousarray(blocks, dtype=np.int32)
        loss = ctypes.c_double()
        g = np.zeros(NET_PARAMS, dtype=np.float32)
        self._ck(self.lib.ggf_net_loss_grad(self.h, len(th), th.ctypes.data, bl.ctypes.data, ctypes.byref(loss),
                                            g.ctypes.data))
        return loss.value, g

    def train(self, theta_dev, batch, n_steps, lr):
        """Adam steps on a device tensor of configurations [n_cfg, 2L^2]."""
        losses = np.zeros(int(n_steps), dtype=np.float32)
        st = _stream([theta_dev])
        self._ck(self.lib.ggf_net_train(self.h, int(theta_dev.shape[0]), _ptr(theta_dev)[0], int(batch), int(n_steps),
                                        float(lr), losses.ctypes.data, st))
        return losses


def sample_group(ctxs, n_sweeps):
    """Sweep several contexts as one graph launch per sweep; returns their
    observables (numpy, [n_sweeps, n_chains, 3] each)."""
    lib = load()
    n = len(ctxs)
    handles = (ctypes.c_void_p * n)(*[c.h.value for c in ctxs])
    outs = [np.zeros((int(n_sweeps), c.n_chains, N_OBS)) for c in ctxs]
    ptrs = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
    st = lib.ggf_sample_group(handles, n, int(n_sweeps), ptrs, MEM_HOST, None)
    if st != 0:
        msgs = "; ".join(lib.ggf_last_error(c.h).decode() for c in ctxs)
        raise GGFError(st, msgs)
    return outs


def _torch_like(t, shape):
    import torch
    return torch.zeros(shape, dtype=torch.float64, device=t.device)
