"""Writes z4_noise.json: the first 64 Z4 codes of three (noise id, config id)
pairs, from the oracle's Philox4x32-10 noise (oracle/noise.py).  The codes are
pinned to the published Philox known-answer vectors through the same
generator; this file freezes the index order (t, alpha, n) and seed rule."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.noise import z4_codes  # noqa: E402

cases = []
for (s, k, nt, nv) in [(0, 1000, 8, 8), (1, 1001, 32, 32), (65535, 65535, 128, 64)]:
    c = z4_codes(nt, nv, s, k)
    cases.append({"noise_id": s, "config_id": k, "nt": nt, "nv": nv, "first64": c.ravel()[:64].tolist()})
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "z4_noise.json"), "w") as f:
    json.dump({"written_by": "tests/golden/make_z4_golden.py (oracle only)", "cases": cases}, f, indent=1)
