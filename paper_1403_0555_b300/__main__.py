"""Command line: enumerate the Gribov copies of one synthetic orbit.

    python -m paper_1403_0555_b300 enumerate --dim 4 --L 4 --kappa 0.714 --seed 2 \\
        --starts 65536 --precision mixed
    python -m paper_1403_0555_b300 tables --entries 2:4,4:2 --orbits 100 --mebisamples 4
    python -m paper_1403_0555_b300 section4 --entries 2:6,3:4 --orbits 100 --mebisamples 4
    python -m paper_1403_0555_b300 section4 --compare 2:10 --orbits 10 --mebisamples 4 \\
        --large-mebisamples 256

`enumerate` prints the orbit's statistics as one JSON line; `tables` one line
per lattice of paper-style statistics over random uniform orbits (the number
of minima of Table I, the global-minimum functional of Table III and the
discovery curve of Figs. 1-3).  `section4` prints per lattice the global
minima (Table III), the relative deviation of the minima from them (Fig. 8)
and the normalised distribution of the functional (Fig. 7); with --compare,
the bin-by-bin comparison of two sample sizes (Fig. 5).  Orbits are seeded synthetic
inputs (orbit_inputs): von Mises(kappa) link angles, or uniform with --kappa 0.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import orbit_inputs as oi
    import paper_1403_0555_b300 as gb

    p = argparse.ArgumentParser(prog="python -m paper_1403_0555_b300")
    sub = p.add_subparsers(dest="cmd", required=True)
    e = sub.add_parser("enumerate", help="enumerate the copies of one synthetic orbit")
    e.add_argument("--dim", type=int, default=4)
    e.add_argument("--L", type=int, default=4)
    e.add_argument("--kappa", type=float, default=1.0, help="von Mises concentration; 0 = uniform")
    e.add_argument("--seed", type=int, default=1, help="orbit seed (also the orbit id)")
    e.add_argument("--starts", type=int, default=65536)
    e.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    e.add_argument("--omega", type=float, default=1.7)
    e.add_argument("--eps", type=float, default=1e-24)
    e.add_argument("--check-every", type=int, default=None)
    e.add_argument("--max-sweeps", type=int, default=None, help="sweep cap per start (library default if unset)")
    e.add_argument("--fp-mode", choices=["auto", "lanczos", "dense", "none"], default="auto")
    t = sub.add_parser("tables", help="paper-style statistics over random uniform orbits "
                                      "(number of minima, global-minimum F/(dV), discovery curve)")
    t.add_argument("--entries", default="2:2,2:4,3:2,4:2", help="comma list of d:N")
    t.add_argument("--orbits", type=int, default=100)
    t.add_argument("--mebisamples", type=float, default=4.0, help="starts per orbit / 1024^2")
    t.add_argument("--omega", type=float, default=1.0)
    t.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    s4 = sub.add_parser("section4", help="distribution of the functional at the minima (Section IV)")
    s4.add_argument("--entries", default="2:4,3:4", help="comma list of d:N")
    s4.add_argument("--compare", default=None, help="d:N: compare two sample sizes bin by bin instead")
    s4.add_argument("--orbits", type=int, default=100)
    s4.add_argument("--mebisamples", type=float, default=4.0, help="starts per orbit / 1024^2")
    s4.add_argument("--large-mebisamples", type=float, default=256.0, help="the larger run of --compare")
    s4.add_argument("--omega", type=float, default=1.0)
    s4.add_argument("--width", type=float, default=1e-3, help="bin width of the distribution")
    a = p.parse_args(argv)
    if a.cmd == "section4":
        from paper_1403_0555_b300.analysis import compare_sample_sizes, section_iv_statistics
        n = int(a.mebisamples * (1 << 20))
        if a.compare:
            d, N = (int(x) for x in a.compare.split(":"))
            print(json.dumps(compare_sample_sizes(d, N, a.orbits, n, int(a.large_mebisamples * (1 << 20)),
                                                  a.omega)), flush=True)
            return
        for ent in a.entries.split(","):
            d, N = (int(x) for x in ent.split(":"))
            print(json.dumps(section_iv_statistics(d, N, a.orbits, n, a.omega, width=a.width)), flush=True)
        return
    if a.cmd == "tables":
        from paper_1403_0555_b300.analysis import table_statistics
        for ent in a.entries.split(","):
            d, N = (int(x) for x in ent.split(":"))
            st = table_statistics(d, N, a.orbits, int(a.mebisamples * (1 << 20)), a.omega,
                                  gb.GC_MIXED if a.precision == "mixed" else gb.GC_FP64,
                                  check_every=4 if a.precision == "mixed" else 1, curve=True)
            print(json.dumps(st), flush=True)
        return

    d, L = a.dim, a.L
    phi = (oi.uniform_orbit(d, L, a.seed) if a.kappa == 0
           else oi.von_mises_orbit(d, L, a.kappa, a.seed))
    mixed = a.precision == "mixed"
    opt = gb.gc_options_default(
        precision=gb.GC_MIXED if mixed else gb.GC_FP64,
        check_every=a.check_every or (4 if mixed else 1),
        **({} if a.max_sweeps is None else {"max_sweeps": a.max_sweeps}),
        fp_mode={"auto": 0, "lanczos": 1, "dense": 2, "none": 3}[a.fp_mode])
    h = gb.gc_create_orbit(d, L, phi, a.seed)
    try:
        gb.gc_enumerate_copies(h, a.starts, a.omega, a.eps, opt)
        st = gb.gc_orbit_stats(h)
    finally:
        gb.gc_destroy_orbit(h)
    print(json.dumps({"dim": d, "L": L, "kappa": a.kappa, "seed": a.seed, "starts": a.starts,
                      "precision": a.precision, **st}))


if __name__ == "__main__":
    main()
