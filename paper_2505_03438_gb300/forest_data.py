"""Training data of the Random Forest strategy (Sec. 5.3), measured on the
GPU the library runs on: for every synthetic scenario of
`scenarios.training_scenarios`, after 60 steps (so that the tuning phase
weights the build times by the rebuild interval the displacements allow),
the live statistics (Sec. 4) and the cost per step of every default
candidate configuration from one full-search tuning phase (each trial
rebuilds and advances `trial_steps` steps, the paper's trials being ten
iterations with one build).

    python -m paper_2505_03438_gb300.forest_data OUT.jsonl
"""
import json
import sys
import time

from . import scenarios
from .forest import DEFAULT_DATA, FEATURES


def collect(out_path=DEFAULT_DATA, trial_steps=10, seed=7, log=print):
    import paper_2505_03438_gb300 as lj

    t0 = time.time()
    with open(out_path, "w") as f:
        for sc in scenarios.training_scenarios(seed):
            s = lj.System(sc)
            try:
                # enough steps for the tuning phase to observe how often the
                # displacements force a rebuild
                s.step(60)
                st = s.stats()
                s.autotune(strategy="full", trial_steps=trial_steps)
                costs = {name: cost for name, (cost, _) in lj.ljsel_tuner_costs(s.h).items()}
            finally:
                s.close()
            rec = dict(name=sc["name"], n=len(sc["x"]), features=[float(st[k]) for k in FEATURES], costs=costs)
            f.write(json.dumps(rec) + "\n")
            f.flush()
            best = min(costs.items(), key=lambda kv: kv[1])
            log("%-20s N=%7d skin %.1f best %s %.4f ms (%.0f s)" % (sc["name"], rec["n"], sc["skin"], best[0], best[1],
                                                                  time.time() - t0))


if __name__ == "__main__":
    collect(sys.argv[1] if len(sys.argv) > 1 else DEFAULT_DATA)
