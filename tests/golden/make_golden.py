"""Writes closed_forms.json: exact expected values for small axis-aligned
voxel stacks (Eq. 5-6 of arXiv 2202.05628, exclusive transmittance, early stop
after the hit at which T falls below tau).

The values come from sympy in exact arithmetic, evaluated to 30 digits; this
script does not call the oracle.  A ray along a coordinate axis through voxel
centres crosses each voxel of the stack over one full side h.
"""
import json
import os

import sympy as sp

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.json")


def case(name, depth, ijk, features, density, direction, tau, note):
    h = sp.Rational(1, 2 ** depth)
    origin = sp.Rational(-1, 2)
    axis = [i for i, v in enumerate(direction) if v != 0][0]
    sign = 1 if direction[axis] > 0 else -1
    # order of traversal along the axis
    order = sorted(range(len(ijk)), key=lambda i: sign * ijk[i][axis])
    C = len(features[0])
    F = [sp.Integer(0)] * C
    optical = sp.Integer(0)
    used = 0
    for i in order:
        s = sp.nsimplify(density[i])
        T = sp.exp(-optical)
        a = 1 - sp.exp(-s * h)
        for c in range(C):
            F[c] += T * a * sp.nsimplify(features[i][c])
        optical += s * h
        used += 1
        if sp.N(sp.exp(-optical), 40) < tau:
            break
    first = order[0]
    target = [float(origin + (sp.Integer(ijk[first][a]) + sp.Rational(1, 2)) * h) for a in range(3)]
    return dict(name=name, note=note, depth=depth, ijk=ijk, features=features, density=density,
                direction=direction, target=target, dist=0.75, tau=tau,
                F=[float(sp.N(v, 30)) for v in F], A=float(sp.N(1 - sp.exp(-optical), 30)),
                order=order[:used] + order[used:], used=used)


cases = [
    case("single", 4, [[8, 8, 8]], [[0.5, -1.25, 2.0]], [3.0], [0, 0, 1], 1e-4,
         "F = (1 - e^{-sigma h}) f, A = 1 - e^{-sigma h}"),
    case("stack3_z", 5, [[10, 11, 4], [10, 11, 5], [10, 11, 6]],
         [[1.0, 0.0], [0.0, 1.0], [-0.5, 0.25]], [7.0, 2.5, 40.0], [0, 0, 1], 1e-4,
         "three voxels in front-to-back order along +z"),
    case("stack3_negz", 5, [[10, 11, 4], [10, 11, 5], [10, 11, 6]],
         [[1.0, 0.0], [0.0, 1.0], [-0.5, 0.25]], [7.0, 2.5, 40.0], [0, 0, -1], 1e-4,
         "the same stack seen from -z: order reversed"),
    case("stack_x_stop", 3, [[2, 3, 3], [3, 3, 3], [4, 3, 3]],
         [[0.375], [0.75], [0.875]], [40.0, 40.0, 5.0], [1, 0, 0], 1e-4,
         "opaque pair along +x: the stop fires after the second hit (features exact in FP32)"),
]
with open(OUT, "w") as fh:
    json.dump({"source": "arXiv 2202.05628 Eq. 5-6 (exclusive T), early stop once T < tau; exact sympy",
               "cases": cases}, fh, indent=1)
print("wrote", OUT)
