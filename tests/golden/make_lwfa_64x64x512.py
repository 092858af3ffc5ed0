"""Writes the FP64 oracle's reference summaries of the boosted laser-wakefield stage on a
downscaled grid: the recipe of tests/synth.py lwfa_stage (cell size, laser, plasma at
n/n_c = 1/900 with its ion background, order-2 shape, 3-pass filter, Vay pusher,
absorbing box) on 64 x 64 x 512 cells with 4 electrons per cell (8,388,608 particles), for
gamma_boost in {2, 5, 13, 30, 100} (SplitMix64 seed 4 + the boost's index), 100 steps.

Calls only the oracle (oracle/), never the CUDA library.  For each boost it stores, at
steps 50 and 100, the wake field E_z and the laser field E_x along the axis (node 32, 32
in x and y), the root-mean-square of E_z over each z plane, and every 10 steps the field
and kinetic energies, the total charge and the particle counts, in
lwfa_64x64x512_gb<gamma>.json beside this script.  One process per boost; a run takes
about two hours on one core.

    python tests/golden/make_lwfa_64x64x512.py [gamma ...]
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

GAMMAS = (2.0, 5.0, 13.0, 30.0, 100.0)
GRID = (64, 64, 512)
PPC = 4
STEPS = 100
CHECKPOINTS = (50, 100)
DIAG_EVERY = 10
AXIS = (32, 32)


def golden_path(gb):
    return os.path.join(HERE, f"lwfa_64x64x512_gb{gb:g}.json")


def run(gb):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np

    import oracle
    import synth

    seed = 4 + GAMMAS.index(gb)
    w = synth.lwfa_stage(GRID, gb, PPC, seed=seed)
    s = oracle.Sim(3, w["n"], (1, 1, 1), w["dx"], w["dt"], order=2, filter_passes=3, tile=(8, 8, 8))
    p = w["plasma"]
    s.load_lab_frame(gb, laser=w["laser"], plasma=[p[0], p[1], p[2], p[3], *p[4], p[5]])
    out = {"gamma_boost": gb, "grid": list(GRID), "ppc": PPC, "seed": seed, "dx": list(w["dx"]), "dt": w["dt"],
           "axis": list(AXIS), "particles_loaded": s.num_particles(), "diagnostics": [], "checkpoints": {}}
    t0 = time.time()
    for n in range(STEPS + 1):
        if n > 0:
            s.step(1)
        if n % DIAG_EVERY == 0:
            d = s.diagnostics()
            out["diagnostics"].append({"step": n, "field_energy": d["field_energy"],
                                       "kinetic_energy": d["kinetic_energy"], "total_charge": d["total_charge"],
                                       "n_particles": d["n_particles"], "n_lost": d["n_lost"]})
        if n in CHECKPOINTS:
            ez = s.get_field(oracle.EZ)
            ex = s.get_field(oracle.EX)
            out["checkpoints"][str(n)] = {
                "ez_axis": ez[:, AXIS[1], AXIS[0]].tolist(),
                "ex_axis": ex[:, AXIS[1], AXIS[0]].tolist(),
                "ez_plane_rms": np.sqrt((ez ** 2).mean(axis=(1, 2))).tolist(),
            }
            print(f"gamma_b {gb:g}: step {n} after {time.time() - t0:.0f} s", flush=True)
    out["oracle_seconds"] = time.time() - t0
    with open(golden_path(gb), "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")
    return gb


if __name__ == "__main__":
    gammas = [float(g) for g in sys.argv[1:]] or list(GAMMAS)
    sys.path.insert(0, ROOT)
    import oracle

    oracle.build()
    with mp.get_context("spawn").Pool(len(gammas)) as pool:
        for gb in pool.imap_unordered(run, gammas):
            print(f"wrote {golden_path(gb)}", flush=True)
