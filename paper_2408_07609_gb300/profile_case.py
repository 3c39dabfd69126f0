"""A small launch of the step kernel for profilers.

    python -m paper_2408_07609_gb300.profile_case [fp32|fp64] [warm] [steps] [ring|full]

builds the 4-level serving hierarchy (7.95 M cells, seed 5; state larger than L2 but
well under a GB) and steps it `warm` then `steps` times with one launch per step, so a
profiler can skip the warm launches and capture single-step launches. `full` selects
full fine-to-coarse feedback (default: ring).
"""
import sys

from . import rti
from . import scenarios as S


def main(argv):
    prec = rti.FP64 if (argv[1:2] or ["fp32"])[0] == "fp64" else rti.FP32
    warm = int(argv[2]) if len(argv) > 2 else 3
    steps = int(argv[3]) if len(argv) > 3 else 2
    fb = rti.NEST_FULL if (argv[4:5] or ["ring"])[0] == "full" else rti.NEST_RING
    sc = S.serving_hierarchy("4level", seed=5, hours=0.01)
    h = rti.Handle.from_scenario(sc, precision=prec, schedule=rti.SCHED_PER_PASS,
                                 nest_feedback=fb)
    h.step(warm)
    h.sync()
    h.step(steps)
    h.sync()
    print("cells", sc.cells, "steps", warm + steps)
    h.close()


if __name__ == "__main__":
    main(sys.argv)
