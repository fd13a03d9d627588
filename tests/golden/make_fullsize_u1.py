"""Write u1_16x16_nv2_k2.json: the oracle's log N(G) and per-pair log N_nm(G)
for one seeded 16 x 16 U(1) configuration with n_v = 2 and K = 2 (Sec. 5;
the covariance route on the full physical + virtual space, 4608 x 4608).

Calls only oracle/ and the seeded input generator; takes a few minutes.
    python tests/golden/make_fullsize_u1.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import ggf_inputs as gi  # noqa: E402
from oracle import weight  # noqa: E402
from oracle.weight import combine  # noqa: E402

SEED, BOND_SCALE, LINKS_SEED = 20241202, 0.3, 1616


def main():
    p = gi.make_problem(16, gi.U1, 2, 2, seed=SEED, bond_scale=BOND_SCALE)
    links = gi.random_links(p, 1, seed=LINKS_SEED)[0]
    W = weight.Weights(p)
    lnm = W.log_n_matrix(links)
    out = {
        "what": "oracle log N(G) and log N_nm(G) (re, im) of gi.random_links(p, 1, seed=links_seed)[0] for "
                "gi.make_problem(16, U1, 2, 2, seed, bond_scale)",
        "seed": SEED, "bond_scale": BOND_SCALE, "links_seed": LINKS_SEED,
        "log_norm": combine(lnm, p.lam),
        "log_n_nm": {f"{n}{m}": [lnm[n, m].real, lnm[n, m].imag] for n in range(2) for m in range(2)},
    }
    with open(os.path.join(HERE, "u1_16x16_nv2_k2.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
