"""Writes the brute-force HMM fixtures in this folder.  Calls only ``oracle.brute``.

Fixture hmm_k2_t5.json: a 2-state, 3-symbol HMM with an asymmetric transition matrix
(so a transposed A or a swapped index changes the answer), observation sequence of
length 5; its log-likelihood and expected counts by enumeration of all 2^5 state paths
(forward algorithm / forward-backward textbook definitions; the paper is silent on HMMs
and uses them nowhere -- the recursion is a map-of-reduce inside a sequential loop,
Appendix A, Fig. "pmexpr-extension").

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import brute  # noqa: E402

CASES = {
    "hmm_k2_t5": {
        "A": [[0.7, 0.3], [0.1, 0.9]],
        "B": [[0.5, 0.4, 0.1], [0.1, 0.3, 0.6]],
        "pi": [0.6, 0.4],
        "obs": [0, 2, 1, 2, 0],
    },
    "hmm_k3_t4": {
        "A": [[0.2, 0.5, 0.3], [0.6, 0.1, 0.3], [0.25, 0.25, 0.5]],
        "B": [[0.9, 0.1], [0.2, 0.8], [0.5, 0.5]],
        "pi": [0.5, 0.3, 0.2],
        "obs": [1, 0, 0, 1],
    },
}


def main():
    for name, c in CASES.items():
        ll, xi, cnt, g1 = brute.expected_counts(c["A"], c["B"], c["pi"], c["obs"])
        out = dict(c)
        out.update(source="oracle.brute enumeration over all K^T state paths",
                   loglik=ll, xi=xi.tolist(), counts=cnt.tolist(), gamma1=g1.tolist())
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
