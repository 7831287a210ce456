"""Write ``oracle_values.json``: FP64 oracle results for the benchmark workloads.

Calls only ``oracle/`` and the workload parameters in ``workloads/``; the CUDA
library is never imported.  Each classical entry holds ln Z / N after the
workload's step count, the free energy per site, and the per-step ln c_n,
discarded weights, side and normalised spectrum head of the chosen
environment; each quantum-chain entry (D_cut <= 32) holds ln Z / N_cells and
the free energy per site of the whole schedule; ``sweep_subset16`` holds
ln Z / N of each instance of the seeded 16-instance subset of the batched
sweep.

    python tests/golden/make_oracle_values.py [name ...]

Entries already present are kept unless named on the command line.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import heisenberg, hotrg  # noqa: E402
from workloads import CONFIGS, QUANTUM_CONFIGS, sweep_subset  # noqa: E402

OUT = os.path.join(HERE, "oracle_values.json")


def initial(cfg):
    if cfg.family == "ising":
        return hotrg.ising_initial_tensor(cfg.beta, cfg.h)
    return hotrg.potts_initial_tensor(cfg.q, cfg.beta)


def compute(cfg):
    t0 = time.time()
    r = hotrg.run(initial(cfg), cfg.D_cut, cfg.steps)
    lz = r.ln_z_per_site
    return {
        "family": cfg.family, "beta": cfg.beta, "h": cfg.h, "q": cfg.q, "D_cut": cfg.D_cut,
        "steps": cfg.steps, "first": "x",
        "ln_z_per_site": lz, "free_energy": -lz / cfg.beta,
        "per_step": [{"dir": s.direction, "Dx": s.Dx, "Dy": s.Dy, "Dn": s.Dn, "ln_c": s.ln_c,
                      "eps_L": s.eps_L, "eps_R": s.eps_R, "side": s.side,
                      "cut_gap": s.cut_gap if s.cut_gap != float("inf") else None,
                      "trace_G": s.trace_G, "spectrum_head": [float(v) for v in s.spectrum[:8]]}
                     for s in r.steps],
        "oracle_seconds": time.time() - t0,
    }


def compute_quantum(q):
    t0 = time.time()
    r = heisenberg.run(heisenberg.cell_tensor(q.Jxy, q.Jz, q.tau), q.D_cut, q.n_time, q.n_space)
    lz = r.ln_z_per_site
    return {
        "family": "xxz_chain", "Jxy": q.Jxy, "Jz": q.Jz, "tau": q.tau, "beta": q.beta,
        "n_time": q.n_time, "n_space": q.n_space, "D_cut": q.D_cut,
        "ln_z_per_site": lz, "free_energy": heisenberg.free_energy_per_site(lz, q.tau),
        "min_cut_gap": min([s.cut_gap for s in r.steps if s.Dn < s.Dx * s.Dx] or [None]),
        "oracle_seconds": time.time() - t0,
    }


def compute_sweep_subset():
    """ln Z / N of the 16-instance subset of the batched sweep (4 per cut group,
    25 steps each), with each run's smallest relative gap at the cut."""
    t0 = time.time()
    rows = []
    for m in sweep_subset():
        r = hotrg.run(hotrg.ising_initial_tensor(m.beta, m.h), m.D_cut, m.steps)
        gaps = [s.cut_gap for s in r.steps if s.cut_gap != float("inf")]
        rows.append({"name": m.name, "beta": m.beta, "h": m.h, "D_cut": m.D_cut, "steps": m.steps,
                     "ln_z_per_site": r.ln_z_per_site, "min_cut_gap": min(gaps) if gaps else None})
        print(f"  {m.name} D_cut={m.D_cut} beta={m.beta:.6f}: ln Z/N = {r.ln_z_per_site:.16f}", flush=True)
    return {"instances": rows, "first": "x", "oracle_seconds": time.time() - t0,
            "ln_z_per_site": rows[0]["ln_z_per_site"]}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    every = (list(CONFIGS) + [n for n in QUANTUM_CONFIGS if QUANTUM_CONFIGS[n].D_cut <= 32]
             + ["sweep_subset16"])
    todo = names or [n for n in every if n not in data]
    for name in todo:
        print(f"oracle: {name} ...", flush=True)
        if name == "sweep_subset16":
            data[name] = compute_sweep_subset()
        else:
            data[name] = compute(CONFIGS[name]) if name in CONFIGS else compute_quantum(QUANTUM_CONFIGS[name])
        print(f"  ln Z/N = {data[name]['ln_z_per_site']:.16f} ({data[name]['oracle_seconds']:.0f} s)", flush=True)
        json.dump(data, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
