"""One synthetic determinant job through the plain and the batched forms,
checked equal: a small self-contained workload for profiling one kernel, e.g.

    python -m paper_2010_12117_gb300.case --n 24 --degs 3,3

runs condense_kernel<24, ...> on 73 x 73 nodes per prime (plain form, then
the batched form in the chosen mode) and prints the job's sizes.  Other
stages: ``--stage eval`` / ``--stage crt`` run one stage alone on inputs
larger than L2, and ``--stage batched`` runs one profiled step of the
256-matrix batched workload (between cudaProfilerStart and Stop);
``--stage probe`` runs the integer-pipe probes of polydet_probe_int_peaks.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=24)
    ap.add_argument("--degs", default="3,3", help="entry degree per variable, comma separated")
    ap.add_argument("--density", type=float, default=0.7)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--mode", choices=("default", "fused", "materialized"), default="default")
    ap.add_argument("--chunk-words", type=int, default=0, help="materialized chunk budget (0: default)")
    ap.add_argument("--stage", choices=("det", "eval", "crt", "batched", "probe"), default="det",
                    help="det: the whole job in both forms; eval: the evaluation of the 12x12 "
                         "trivariate workload alone; crt: the CRT of 2^24 coefficients alone; "
                         "batched: two steps of the 256-matrix batched workload (seed 0, the "
                         "autotuner's cached choices, CUDA graphs), the second between "
                         "cudaProfilerStart and cudaProfilerStop; probe: the integer-pipe probes")
    ap.add_argument("--primes", type=int, default=5, help="primes for --stage eval / crt")
    ap.add_argument("--full-grid", action="store_true", help="--stage eval on the power-of-two grid")
    args = ap.parse_args(argv)

    import torch
    if args.stage == "batched":
        return _batched()
    if args.stage == "probe":
        from paper_2010_12117_gb300 import binding
        imad, upd, pair, triple = binding.probe_int_peaks()
        print(f"ok probes: {imad:.4g} IMAD/s, {upd:.4g} single-step updates/s, "
              f"{pair:.4g} two-step element updates/s, {triple:.4g} three-step element updates/s")
        return 0
    if args.stage != "det":
        return _stage(args)
    from . import synth
    from .binding import BATCH_FUSED, BATCH_MATERIALIZED
    from .runner import BatchedRunner, PlainRunner

    degs = tuple(int(x) for x in args.degs.split(","))
    rng = np.random.default_rng(args.seed)
    pm = synth.random_matrix(rng, args.n, degs, args.density, -30000, 30000)
    st = torch.cuda.Stream()
    pr = PlainRunner([pm])
    pr.upload(st)
    pr.compute(st)
    pr.download(st)
    st.synchronize()
    pr.check_status(st)
    want = pr.results()[0]
    pl = pr.plans[0]
    sizes = f"n={args.n} degs={degs} P={pl.P} G={pl.G} coefficients={len(want)}"
    pr.close()

    br = BatchedRunner([pm], tune=False, stream=st)
    if args.mode != "default":
        br.set_modes(BATCH_FUSED if args.mode == "fused" else BATCH_MATERIALIZED)
    if args.chunk_words:
        br.set_chunk_words(args.chunk_words)
    br.upload(st)
    br.compute(st)
    br.download(st)
    st.synchronize()
    br.check_status(st)
    got = br.results()[0]
    br.close()
    if got != want:
        print("MISMATCH between the plain and the batched form", sizes)
        return 1
    print("ok", sizes)
    return 0


def _batched() -> int:
    """One warm step and one profiled step of the batched workload."""
    import torch
    from . import synth
    from .runner import BatchedRunner
    st = torch.cuda.Stream()
    r = BatchedRunner(synth.batched(0, 256), tune="cache", stream=st)
    r.upload(st)
    r.capture(st)
    r.compute(st)
    st.synchronize()
    torch.cuda.profiler.start()
    r.compute(st)
    st.synchronize()
    torch.cuda.profiler.stop()
    r.check_status(st)
    print("ok batched step:", r.modp_dets(), "determinants mod p, modes", r.tuning or "default")
    r.close()
    return 0


def _stage(args) -> int:
    """One stage alone, twice (a warm-up launch and one to profile)."""
    import torch
    from . import synth
    from .binding import Plan
    st = torch.cuda.Stream()
    P = args.primes
    if args.stage == "eval":
        pm = synth.sparse_12x12_xyz(0)
        pl = Plan(pm.n, pm.degs, P, full_grid=args.full_grid)
        c = torch.from_numpy(pm.coeffs.astype(np.int32).reshape(-1)).cuda()
        ev = torch.empty(P * pm.n * pm.n * pl.G, dtype=torch.int32, device="cuda")
        ws = pl.workspace(P)
        for _ in range(2):
            pl.eval(c, 0, P, ev, ws, st)
        sizes = f"eval 12x12 over Z[x,y,z], G={pl.G}, P={P}, {4 * ev.numel() / 1e6:.0f} MB written"
    else:
        pl = Plan(1, (4095, 4095), P)  # C = 4096^2 coefficients
        g = torch.Generator(device="cuda").manual_seed(args.seed)
        res = torch.randint(0, 2 ** 30, (P * pl.C,), dtype=torch.int32, device="cuda", generator=g)
        limbs = torch.empty(pl.C * pl.W, dtype=torch.int32, device="cuda")
        for _ in range(2):
            pl.crt(res, limbs, st)
        sizes = f"crt of C={pl.C} coefficients, P={P}, W={pl.W}"
    st.synchronize()
    pl.close()
    print("ok", sizes)
    return 0


if __name__ == "__main__":
    sys.exit(main())
