"""Time forward advances of one of the library's synthetic workloads with a pinned launch plan.

    python -m paper_2511_09389_gb300.timing --workload paper --sources 256 \\
        --plan 1,32,4,2 --accumulation fixed --calls 3

Each call is one rt_advance on the device-resident inputs; the march kernel's CUDA-event time
(the handle's profile mode) is printed per call. Used to profile one kernel on a bounded case
(a subset of the sources keeps an ncu capture short); the benchmark itself is bench.py.
"""
import argparse
import sys

WORKLOADS = ("turbulent", "paper", "inverse")


def problem(name: str):
    from . import inputs
    if name == "turbulent":
        return inputs.turbulent()
    if name == "paper":
        return inputs.paper_timing()
    if name == "inverse":
        return inputs.inverse_problem()
    raise ValueError(f"workload must be one of {WORKLOADS}")


def run(workload: str, sources: int = 0, plan=None, accumulation: str = "auto", calls: int = 3):
    """Advance `calls` times; return the march kernel's milliseconds per call."""
    import torch
    from .api import Grid
    p = problem(workload)
    src = p.sources if sources <= 0 else p.sources[:sources]
    j, k = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa))
    s = torch.from_numpy(src.copy()).cuda()
    g = Grid(p.shape, p.n_freq, profile=True, plan=plan, accumulation=accumulation)
    out = torch.empty_like(j)
    ms = []
    try:
        for _ in range(calls):
            g.advance(j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step, out=out)
            torch.cuda.synchronize()
            ms.append(g.kernel_ms())
        info = {"plan": g.last_plan(), "accumulation": g.last_accumulation(), "sources": len(src),
                "rays": p.num_rays}
    finally:
        g.close()
    return ms, info


def main(argv=None):
    ap = argparse.ArgumentParser(description="time forward advances of a synthetic workload")
    ap.add_argument("--workload", choices=WORKLOADS, default="turbulent")
    ap.add_argument("--sources", type=int, default=0, help="use the first N sources (0: all)")
    ap.add_argument("--plan", default="", help="'bins_per_group,block,gathers[,lanes_per_ray[,tile]]'")
    ap.add_argument("--accumulation", default="auto", choices=("auto", "fp32", "fp64", "fixed"))
    ap.add_argument("--calls", type=int, default=3)
    a = ap.parse_args(argv)
    plan = tuple(int(x) for x in a.plan.split(",")) if a.plan else None
    ms, info = run(a.workload, a.sources, plan, a.accumulation, a.calls)
    for i, t in enumerate(ms):
        print(f"call {i}: march kernel {t:.4f} ms", flush=True)
    print(info)
    return 0


if __name__ == "__main__":
    sys.exit(main())
