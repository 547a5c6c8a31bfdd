"""Tiny-grid runs shared by the index-check test: every kernel form (one step,
vector access, TMA-staged and two steps per launch; the batch forms; D3Q19) on
grids of 3 to 14 nodes per side (every node is a boundary node or next to one,
or, at 13 and 14 nodes, in the vector form's one interior group per row).  Run as a
script it writes the results to an .npz file, with whatever libbtrt the
BTRT_LIBRARY environment variable selects."""
import sys

import numpy as np

import workloads as w

GRIDS_2D = [(4, 4, (0, 0, 0, 0)), (5, 5, (1, 1, 1, 1)), (7, 3, (0, 0, 1, 1)), (3, 3, (1, 1, 0, 0)),
            (3, 7, (1, 1, 1, 1)), (13, 5, (0, 0, 0, 0)), (14, 6, (1, 1, 1, 1))]
FORMS_2D = [("f64", "f64", "ref", "plain"), ("df64", "df64", "ref", "plain"), ("f32", "f32", "ref", "plain"),
            ("f32", "f16", "local", "plain"), ("f32", "bf16", "ref", "tma"), ("f32", "f16", "local", "tma"),
            ("f32", "f32", "ref", "tb2"), ("f32", "f16", "local", "tb2"), ("f32", "bf16", "ref", "tb2"),
            ("f32", "f32", "ref", "vec"), ("f32", "f16", "local", "vec"), ("f32", "bf16", "local", "vec"),
            ("f32", "f32", "ref", "tb2v"), ("f32", "f16", "local", "tb2v"), ("f32", "bf16", "ref", "tb2v"),
            ("f32", "f32", "local_dw", "plain"), ("f32", "f16", "local_dw", "plain"),
            ("f32", "f16", "local_sr", "plain"), ("f32", "bf16", "local_sr", "vec"),
            ("f32", "bf16", "local_dw_sr", "plain"), ("f32", "bf16", "moment_sr", "plain"),
            ("f32", "f16", "moment_sr", "plain"), ("f32", "f16", "moment_sr", "vec")]
GRIDS_3D = [(3, 3, 3, (0,) * 6), (4, 5, 6, (1,) * 6), (5, 3, 4, (1, 1, 0, 0, 1, 1))]
FORMS_3D = [("f64", "f64", "ref"), ("f32", "f32", "ref"), ("f32", "f16", "local")]


def run_all():
    import torch
    from paper_1902_09813_gb300 import Batch, Lattice, Lattice3
    out, flags = {}, {}
    for gi, (nx, ny, bc) in enumerate(GRIDS_2D):
        for src in ("trig", "const", "reaction"):
            p = w.random_state_problem(nx, ny, seed=gi + 3, bc=bc, nonlinear=True, source=src,
                                       flux_q=2.5 if src == "reaction" else 2.0)
            for comp, st, sh, var in FORMS_2D:
                lat = Lattice.from_problem(p, compute=comp, storage=st, shift=sh)
                if comp == "f32":
                    lat.set_sweep_variant(var)
                lat.init(p.phi0(), t0=p.t0).step(5)
                key = f"2d_{nx}x{ny}_{src}_{comp}_{st}_{sh}_{var}"
                out[key] = lat.phi_host()
                flags[key] = lat.flags()
    # per-node fields
    p = w.variable_tensor(n=6, alpha=1e-2, walls=True, t_end=0.01)
    lat = Lattice.from_problem(p, compute="f64").init(p.phi0()).step(4)
    out["2d_fields"] = lat.phi_host()
    flags["2d_fields"] = lat.flags()
    # a batch of tiny members
    probs = [w.random_state_problem(nx, ny, seed=9 + k, bc=bc) for k, (nx, ny, bc) in enumerate(GRIDS_2D)]
    lats = [Lattice.from_problem(q, compute="f32", storage="f16", stream=torch.cuda.current_stream())
            .init(q.phi0()) for q in probs]
    b = Batch(lats)
    b.step(6, residual=True)
    b.set_tiles(32, 8, 1, 2).step(5, residual=True)   # the two-step batch form, an odd slice
    for k, lt in enumerate(lats):
        out[f"batch_{k}"] = lt.phi_host()
        flags[f"batch_{k}"] = int(b.member_flags()[k])
    b.close()
    for gi, (nx, ny, nz, bc) in enumerate(GRIDS_3D):
        p = w.random_state_problem3(nx, ny, nz, seed=gi + 5, bc=bc, nonlinear=True, source="reaction", flux_q=2.5)
        for comp, st, sh in FORMS_3D:
            lat = Lattice3.from_problem(p, compute=comp, storage=st, shift=sh).init(p.phi0()).step(5)
            key = f"3d_{nx}x{ny}x{nz}_{comp}_{st}_{sh}"
            out[key] = lat.phi_host()
            flags[key] = lat.flags()
    return out, flags


if __name__ == "__main__":
    res, fl = run_all()
    np.savez(sys.argv[1], **res, **{"flags__" + k: np.int32(v) for k, v in fl.items()})
