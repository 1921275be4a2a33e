"""Write the stored results of complete oracle sorts (test fixtures).

Every value written here comes from the CPU oracle (``oracle/``) on the seeded
synthetic inputs of ``paper_2312_13299_gb300.synth``; nothing is read from the
CUDA path.  A fixture records, for one workload, the complete run of the PLAS
schedule (Sec. 3.1) with the default schedule and Philox seed 0:

* the iteration count, the radius levels and the iterations spent at each
  level (the shrink test of Sec. 3.1 decides these);
* the SHA-256 of the final permutation (int32, little endian), of the
  per-iteration fixed-point residual sums (int64) and of the carried
  attributes gathered by the permutation (float32);
* the final schedule state and the two quality objectives of the sorted grid
  (mean L2 distance of 4-neighbours and the mean L2 distance to the last
  target), for the within-1e-4 comparison.

The GPU parity tests must reproduce the hashes bit for bit.  The per-level
iteration counts are also what the CPU baseline of ``bench.py`` multiplies
its per-iteration oracle timings by, so that projection owes nothing to the
CUDA path.

Usage (from the repository root; 512x512 takes about a quarter of an hour on
8 cores, 1024x1024 several hours):

    python tests/golden/make_sort_goldens.py 3dgs-512 [3dgs-1024 ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as orc  # noqa: E402
from paper_2312_13299_gb300 import synth  # noqa: E402

# workload name -> (H, W, generator, data seed)
WORKLOADS = {
    "rgb-64": (64, 64, "rgb", 0),
    "3dgs-512": (512, 512, "3dgs", 0),
    "3dgs-1024": (1024, 1024, "3dgs", 0),
    "rgb-512": (512, 512, "rgb", 0),
}


def fixture_path(name: str) -> str:
    return os.path.join(HERE, f"oracle_sort_{name}.json")


def inputs(name: str):
    H, W, kind, seed = WORKLOADS[name]
    if kind == "rgb":
        return H, W, synth.rgb_uniform(H, W, seed=seed), None
    x, carried = synth.gaussians_3dgs(H * W, seed=seed)
    return H, W, x, carried


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def make(name: str) -> dict:
    H, W, x, carried = inputs(name)
    t0 = time.time()
    r = orc.sort(x, H, W, seed=0, trace_cap=1 << 17)
    secs = time.time() - t0
    st = r["state"]
    it = int(r["iterations"])
    assert len(r["trace_S"]) == it, "trace shorter than the run"
    levels = orc.levels(H, W)
    per_level = np.bincount(r["trace_level"], minlength=len(levels)).astype(int)
    perm = r["perm"]
    sorted_x = orc.gather(x, perm)
    nb_l2, _vad = orc.metrics(sorted_x.reshape(H, W, -1))
    out = {
        "_about": ("complete oracle sort (oracle/plas_oracle.c) of the seeded synthetic "
                   "workload; written by tests/golden/make_sort_goldens.py"),
        "workload": name,
        "H": H, "W": W, "D": int(x.shape[1]),
        "data_seed": WORKLOADS[name][3], "philox_seed": 0,
        "schedule": "default (phi0 = min(H,W)/2 - 1, shrink 0.95, phi_min 1, tol 1e-4, "
                    "sigma_ratio 2, min_block 16, shuffled start, normalised)",
        "iterations": it,
        "levels": int(len(levels)),
        "iterations_per_level": per_level.tolist(),
        "final_state": {"it": int(st.it), "epoch": int(st.epoch), "redraws": int(st.redraws),
                        "level": int(st.level), "done": int(st.done),
                        "d_last": float(st.d_last).hex(), "scale_exp": int(st.scale_exp)},
        "last_trace_S": int(r["trace_S"][-1]),
        "sha256_perm_int32": sha256(perm.astype("<i4")),
        "sha256_trace_S_int64": sha256(r["trace_S"].astype("<i8")),
        "mean_neighbour_l2": float(nb_l2),
        "mean_l2_to_target": float(st.d_last),
        "oracle_seconds": round(secs, 1),
        "oracle_threads": orc.num_threads(),
    }
    if carried is not None:
        out["C"] = int(carried.shape[1])
        out["sha256_carried_out_float32"] = sha256(orc.gather(carried, perm).astype("<f4"))
    return out


def main(argv):
    names = argv or ["3dgs-512"]
    for name in names:
        if name not in WORKLOADS:
            raise SystemExit(f"unknown workload {name}; choose from {sorted(WORKLOADS)}")
        fx = make(name)
        with open(fixture_path(name), "w") as f:
            f.write("{\n" + ",\n".join(f" {json.dumps(k)}: {json.dumps(v)}"
                                        for k, v in fx.items()) + "\n}\n")
        print(f"{name}: {fx['iterations']} iterations over {fx['levels']} levels in "
              f"{fx['oracle_seconds']} s ({fx['oracle_threads']} threads)")


if __name__ == "__main__":
    main(sys.argv[1:])
