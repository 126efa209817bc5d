"""Writes the stored expected values under tests/golden/ from the CPU oracle.

Calls only `oracle` and `workloads` (never the CUDA library).  Each fixture
records its inputs, the oracle settings and the passage it follows.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def square_inclusion():
    ms = W.square_inclusion_15()
    res = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)
    return {
        "citation": "Sec. 5.2 Eq. final_system solved by CG (Sec. 5.3 Lemma); A_H by the "
                    "energy form of Eq. forms_def1; 15x15 grid, central 7x7 inclusion "
                    "(0-based voxels 4..10) of 10*I in 1*I, A0 = I, loads e1, e2",
        "N": list(ms.N),
        "tol": 1e-12,
        "AH": res["AH"].tolist(),
        "iters": res["iters"],
    }


def laminate():
    # closed form: harmonic mean across the layers, arithmetic mean along them
    a = [1.0, 3.0, 10.0, 30.0, 100.0, 30.0, 10.0, 3.0, 1.0]
    harm = len(a) / sum(1.0 / v for v in a)
    arith = sum(a) / len(a)
    return {
        "citation": "exact GaNi solution of a laminate A(x) = a(x_1) I on a 9x7 grid: "
                    "e~ = (harm/a - 1, 0) is curl-free, zero-mean and makes A e constant "
                    "(Sec. 5.2 Eq. GaNiD)",
        "N": [9, 7],
        "layers_axis0": a,
        "AH": [[harm, 0.0], [0.0, arith]],
    }


def circles_729():
    # the 729x729 two-phase workload (40 circles, contrast 100): reference A_H
    # of the oracle at tol 1e-12, used to state the error of the GPU paths
    ms = W.circles_2d()
    res = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)
    return {
        "citation": "Sec. 5.2 Eq. final_system solved by CG (Sec. 5.3 Lemma); A_H by the "
                    "energy form of Eq. forms_def1; workloads.circles_2d() defaults "
                    "(729x729, 40 seeded circles, phases 1*I and 100*I)",
        "N": list(ms.N),
        "tol": 1e-12,
        "vf": ms.meta["vf"],
        "AH": res["AH"].tolist(),
        "iters": res["iters"],
    }


def spheres_135():
    # the 135^3 workload (60 spheres, two random SPD phases, contrast 1000):
    # reference A_H of the oracle at tol 1e-12, against which the GPU paths
    # state their error at this size
    ms = W.spheres_3d()
    res = O.solve_AH(ms.full_field(), ms.N, tol=1e-12)
    return {
        "citation": "Sec. 5.2 Eq. final_system solved by CG (Sec. 5.3 Lemma); A_H by the "
                    "energy form of Eq. forms_def1; workloads.spheres_3d() defaults "
                    "(135^3, 60 seeded spheres, two random SPD phases, contrast 1000)",
        "N": list(ms.N),
        "tol": 1e-12,
        "vf": ms.meta["vf"],
        "AH": res["AH"].tolist(),
        "AH_flux": res["AH_flux"].tolist(),
        "iters": res["iters"],
        "true_rel_res": [float(v) for v in res["true_rel_res"]],
    }


if __name__ == "__main__":
    todo = [("square_inclusion_15.json", square_inclusion), ("laminate_9x7.json", laminate)]
    if "--large" in sys.argv:
        todo.append(("circles_729_AH.json", circles_729))
    if "--large3d" in sys.argv:
        todo = [("spheres_135_AH.json", spheres_135)]
    for name, fn in todo:
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(fn(), f, indent=1)
        print("wrote", name)
