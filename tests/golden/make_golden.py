"""Writes tests/golden/tiny_scene_oracle.json by calling only the oracle.

Regression fixture for the 20,000-Gaussian, 256x256 scene at s_v in {1, 4}:
survivor and pair counts, the frustum max and its argmax, and SHA-256 digests
of the sorted keys/values, the tile ranges and the FP32 image.  Run from the
repository root:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O                       # noqa: E402
from paper_2510_09997_gb300 import synth as S        # noqa: E402


def digest(a):
    return hashlib.sha256(a.tobytes()).hexdigest()


def main():
    sc = S.tiny_scene()
    out = {}
    for s in (1.0, 4.0):
        v = S.tiny_view(s)
        fr = O.frame(sc, [v], with64=False)
        s1 = fr["s1"][0]
        out["s=%g" % s] = dict(
            mask=int(s1["mask"].sum()), survivors=int(s1["survive"].sum()), pairs=int(len(fr["keys"])),
            dmax_bits=int(s1["dmax"].view("uint32")[0]), argmax=int(s1["argmax"][0]),
            keys=digest(fr["keys"]), vals=digest(fr["vals"]), ranges=digest(fr["ranges"]),
            img32=digest(fr["img"][0]["img32"]), ncontrib=digest(fr["img"][0]["ncontrib"]))
    path = os.path.join(ROOT, "tests", "golden", "tiny_scene_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
