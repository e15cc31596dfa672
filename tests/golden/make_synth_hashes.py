"""Writes synth_hashes.txt: SHA-256 of small crops of each seeded generator.

The generators use only correctly rounded IEEE operations, so these hashes
must hold on every host; the test that reads them checks that.  Run from
the repository root:  python tests/golden/make_synth_hashes.py
"""
import hashlib
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from paper_2005_08713_gb300 import synth  # noqa: E402

CASES = [
    ("stain", lambda: synth.stain(synth.config_seed(1), 96, 80)),
    ("slide", lambda: synth.slide(synth.config_seed(3), 12345, 6789, 100, 70)),
    ("phantom", lambda: synth.phantom(synth.config_seed(2), 2048, 2048, 1000, 1000, 90, 60)),
]


def digests():
    return {name: hashlib.sha256(fn().tobytes()).hexdigest() for name, fn in CASES}


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "synth_hashes.txt")
    with open(out, "w") as f:
        f.write("# generator crop -> sha256 of its bytes (written by make_synth_hashes.py)\n")
        for k, v in digests().items():
            f.write(f"{k} {v}\n")
