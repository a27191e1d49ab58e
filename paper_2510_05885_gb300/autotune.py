"""Autotuner of the library's runtime cut-overs, per size class.

For one representative system of a size class (a form, a range of
dimensions, a range of instance counts) it times the factor + refined solve
of every candidate setting of

  persistent_fronts   one persistent launch per level for the large fronts,
                      or one launch per 128-column panel step
  subtree_sweeps      the small subtrees factored and swept by one CTA /
                      warp each, or level launches for every supernode
  tc_min_pivots       the front size from which the FP32 path uses the
                      tensor cores (split TF32) for the dense updates

on the GPU, with the handle's own CUDA-graph replay as in production, and
writes the fastest setting as one line of a table that
``ncl_kkt_options.autotune_path`` points at.  Every candidate is a handle on
the SAME analysis (``ncl_kkt_analyze_like``), so only the numeric phase is
compared, and every candidate's solution is checked against the backward-
error target before it may win.

  python -m paper_2510_05885_gb300.autotune --out tuned.txt [--classes ...]
"""
from __future__ import annotations

import argparse
import itertools
import os
import statistics
import sys

import numpy as np

from . import ncl_kkt as nk
from . import synth

# the default candidate grid
PERSISTENT = (1, 0)
SUBTREE = (1, 0)
TC_MIN = (128, 256, 512)

# size classes: (name, form, dim_lo, dim_hi, count_lo, count_hi, generator)
# dim_hi is exclusive; a generator returns (patterns, values per draw, nrhs)


def _single(form, side, rho, nrhs=1):
    def gen():
        pat = synth.make_pattern(side, side)
        name = "condensed" if form == 1 else "stabilized"
        draws = [synth.draw_instance(pat, np.random.Generator(np.random.PCG64(synth.seed_for(9, d))), form=name,
                                     rho=rho, nrhs=nrhs) for d in range(2)]
        return [pat], [[i] for i in draws], nrhs
    return gen


def _batch(count, side, nrhs):
    def gen():
        rng = np.random.Generator(np.random.PCG64(synth.seed_for(9, 77)))
        E = len(synth.grid_edges(side, side))
        pats = [synth.make_pattern(side, side, np.sort(rng.choice(E, size=int(rng.integers(1, 4)), replace=False)))
                for _ in range(count)]
        draws = [[synth.draw_instance(p, rng, form="stabilized", rho=1e4, nrhs=nrhs) for p in pats] for _ in range(2)]
        return pats, draws, nrhs
    return gen


def _mixed(count, lo, hi):
    def gen():
        sides = synth.adjoint_sides(count, lo, hi)
        cache = {}
        pats = []
        for s in sides:
            s = int(s)
            if s not in cache:
                cache[s] = synth.make_pattern(s, s)
            pats.append(cache[s])
        rng = np.random.Generator(np.random.PCG64(synth.seed_for(9, 78)))
        draws = [[synth.draw_instance(p, rng, form="stabilized", rho=1e4) for p in pats] for _ in range(2)]
        return pats, draws, 1
    return gen


CLASSES = {
    # the configurations of the benchmark's workloads, one class each
    "condensed-300": (1, 100_000, 1_000_000, 1, 1, _single(1, 300, 1e5)),
    "condensed-small": (1, 0, 100_000, 1, 1, _single(1, 96, 1e5)),
    "stabilized-700": (0, 1_000_000, 1 << 40, 1, 1, _single(0, 700, 1e6)),
    "stabilized-tiny": (0, 0, 20_000, 1, 1, _single(0, 22, 1e4)),
    "stabilized-small": (0, 20_000, 1_000_000, 1, 1, _single(0, 150, 1e4)),
    "batch-64x100": (0, 0, 1 << 40, 2, 128, _batch(64, 100, 4)),
    "batch-256-mixed": (0, 0, 1 << 40, 129, 1 << 20, _mixed(256, 10, 70)),
}


def _device_draws(draws, dev):
    import torch
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    out = []
    for insts in draws:
        B = np.concatenate([i.b for i in insts], axis=0)
        out.append(dict(H=T(np.concatenate([i.H_val for i in insts])), J=T(np.concatenate([i.J_val for i in insts])),
                        S=T(np.concatenate([i.Sigma for i in insts])), Bc=T(B.T.copy()),
                        delta=[i.delta for i in insts], rho=[i.rho for i in insts]))
    return out


def time_setting(base, setting, dd, nrhs, reps=7, warm=3):
    """Median device time (ms) of factor + refined solve with ``setting``,
    on a handle sharing ``base``'s analysis; None if the solve misses its
    backward-error target or fails."""
    import torch
    K = nk.KKT.like(base, prec="fp32_ir", **setting)
    try:
        Xc = torch.empty_like(dd[0]["Bc"])
        Bf = torch.empty_like(dd[0]["Bc"])
        flush = torch.empty(64 << 20, dtype=torch.float32, device=Bf.device)   # 256 MB, more than the L2
        times = []
        for i in range(warm + reps):
            d = dd[i % len(dd)]
            Bf.copy_(d["Bc"])
            flush.zero_()      # every timed call starts with a cold L2, as in the benchmark
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            infos, si = nk.ncl_kkt_batch_factor_solve(K._h, d["H"], d["J"], d["S"], d["delta"], d["rho"], nrhs, Bf,
                                                      K.dim, Xc, K.dim)
            e1.record()
            e1.synchronize()
            if si.status != 0 or not si.backward_err <= 1e-10:
                return None
            if i >= warm:
                times.append(e0.elapsed_time(e1))
        return statistics.median(times)
    except nk.NclError:
        return None
    finally:
        K.close()


def tune_class(name, dev="cuda:0", grid=None, log=print):
    form, dlo, dhi, clo, chi, gen = CLASSES[name]
    pats, draws, nrhs = gen()
    dd = _device_draws(draws, dev)
    if len(pats) == 1:
        p = pats[0]
        base = nk.KKT(form, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp32_ir")
    else:
        base = nk.KKT.batch(form, [(p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind) for p in pats],
                            prec="fp32_ir")
    grid = grid or [dict(persistent_fronts=a, subtree_sweeps=b, tc_min_pivots=c)
                    for a, b, c in itertools.product(PERSISTENT, SUBTREE, TC_MIN)]
    results = []
    for setting in grid:
        ms = time_setting(base, setting, dd, nrhs)
        log(f"  {name}: {setting} -> {('%.3f ms' % ms) if ms is not None else 'rejected'}")
        if ms is not None:
            results.append((ms, setting))
    dim = base.dim
    base.close()
    if not results:
        raise RuntimeError(f"no candidate setting of {name} met the target")
    ms, best = min(results, key=lambda t: t[0])
    d = nk.default_options()
    dflt = dict(persistent_fronts=d.persistent_fronts, subtree_sweeps=d.subtree_sweeps, tc_min_pivots=d.tc_min_pivots)
    default = next((m for m, s in results if s == dflt), None)
    line = (f"{form} {dlo} {dhi} {clo} {chi} {best['persistent_fronts']} {best['subtree_sweeps']} 2 "
            f"{best['tc_min_pivots']}  # {name}: dim {dim}, {ms:.3f} ms"
            + (f" (defaults {default:.3f} ms)" if default is not None else ""))
    return line, results


def write_table(lines, path):
    with open(path, "w") as f:
        f.write("# tuned cut-overs: form dim_lo dim_hi count_lo count_hi persistent_fronts subtree_sweeps "
                "use_tensor_cores tc_min_pivots  # class: measured factor + refined solve\n")
        for ln in lines:
            f.write(ln + "\n")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--classes", nargs="*", default=list(CLASSES))
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    nk.load()
    lines = []
    for name in args.classes:
        line, _ = tune_class(name)
        print(line, flush=True)
        lines.append(line)
    write_table(lines, args.out)


if __name__ == "__main__":
    sys.exit(main())
