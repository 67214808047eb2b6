"""Writes the stored trajectories under tests/golden/ by calling only the CPU oracle.

Each file holds one bound per line (iteration 0 first) for one synthetic workload
and parameter preset; the header lines (starting with '#') state the recipe.
Run:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1710_03732_gb300 import instances as I  # noqa: E402

PRESET = dict(kz=1.0, ky=0.5, kx=1.0, phi_y=0.5, phi_z=(0.2,) * 5)


def write(name, inst, iters, dual_mode):
    prm = O.params_array(**PRESET)
    _, lbs, _ = O.run(inst.F, inst.D, inst.B, iters=iters, prm=prm, dual_mode=dual_mode, threads=O.max_threads() or 1)
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        f.write(f"# workload: {inst.name}: {inst.recipe}\n")
        f.write(f"# preset: {PRESET}; dual_mode={dual_mode}; S1 iterations={iters}\n")
        f.write("# source: CPU oracle (oracle/rlt2_oracle.c), FP64, compiled without FMA contraction "
                "(fused multiply-adds only where the oracle calls fma)\n")
        for v in lbs:
            f.write(repr(float(v)) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    write("lb_n8_grid2x4_canonical.txt", I.config(1), 50, 1)
    write("lb_n8_grid2x4_raw.txt", I.config(1), 50, 0)
    write("lb_n12_grid3x4_canonical.txt", I.config(2), 200, 1)
    write("lb_n12_grid3x4_raw.txt", I.config(2), 200, 0)
