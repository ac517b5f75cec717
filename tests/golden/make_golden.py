"""Write tests/golden/tiny_exact.json from the exact oracle only.

Usage:  python tests/golden/make_golden.py
The file holds, for a few seeded tiny hypergraphs (n=12, m=20, rank 4) and a
rational x, the exact y = B x^(N-1) of Eq. (2) evaluated over every entry of
the blowup tensor (Sec. II).  Nothing here touches the CUDA path.
"""
import json
import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import s3synth  # noqa: E402
from oracle import exact  # noqa: E402


def main():
    cases = []
    for seed, N in [(0, 4), (1, 4), (2, 5), (3, 6)]:
        hg = s3synth.tiny_case(seed=seed, rank=4)
        x = [Fraction(1 + (7 * i) % 11, 5 + (3 * i) % 7) for i in range(hg.n)]
        y = exact.ttsv1_bruteforce(hg.n, hg.edges(), x, N)
        cases.append({
            "seed": seed, "N": N, "n": hg.n,
            "edges": [list(e) for e in hg.edges()],
            "x": [str(v) for v in x],
            "y": [str(v) for v in y],
        })
    out = {
        "citation": "Eq. (2) over all entries of the blowup tensor of Sec. II (w(e)=|e|), exact rationals",
        "cases": cases,
    }
    with open(os.path.join(HERE, "tiny_exact.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
