"""The oracle's Woodcock transport against an independent analog transport.

`analog_transport.py` tracks the same pencil beam through a homogeneous water
cube with none of the oracle's machinery: exponential free paths of the local
coefficient instead of Woodcock tracking, Klein-Nishina by rejection from the
uniform law, Thomson by inverting its cumulative, azimuths as angles, new
directions from an explicit frame, numpy's random numbers.  Both must give
the same primary signal and the same scatter image of all orders, ring by
ring, within the statistics of the two runs.  Full-density water 32 mm thick
(0.66 mean free paths at 60 keV) makes multiple scattering, and so the
rotation of directions that are no longer along the beam, part of the image.
A second phantom layers water, a lung-density slice and bone along the beam:
the analog transport integrates the method's trilinear field exactly there
(it is piecewise linear in x), so the mixture, the interaction choice in
mixed regions and the bone-set majorant are checked too.
"""
import math

import numpy as np
import pytest

import oracle
from analog_transport import transport
from paper_1204_6367_gb300 import inputs


@pytest.mark.parametrize("phantom", ["water", "layers"])
def test_woodcock_transport_matches_analog_transport(phantom):
    prob = inputs.uniform_slab_problem(nx=16, ny=16, nz=16, vox=2.0, mat_id=1, density=1.0, energy=60.0,
                                       nu=64, nv=64, det_px=4.0, pencil=True, sdd=1060.0)
    if phantom == "layers":
        # water, a lung-density layer, then bone along the beam: the trilinear
        # mixture blends them between voxel centres, and bone sets the majorant
        prob.density[:, :, 3] = 0.3
        prob.material[:, :, 8:] = 2
        prob.density[:, :, 8:] = 1.85
    n = 2_000_000
    a_prim, a_scat = transport(prob, n, seed=1, half=16.0)
    tp, ts, st, _ = oracle.mc_run(prob, n, seed=3, threads=8)
    o_prim, o_scat = oracle.finalize(tp, n), oracle.finalize(ts, n)
    # primary: binomial counts of 60 keV photons
    c = a_prim.sum() * n / 60.0
    assert o_prim.sum() == pytest.approx(a_prim.sum(), rel=4.0 * math.sqrt(2.0 / c) + 0.002)
    iu, iv = np.meshgrid(np.arange(prob.nu), np.arange(prob.nv))
    rho = np.hypot(iu + 0.5 - (prob.nu // 2 + 0.5), iv + 0.5 - (prob.nv // 2 + 0.5))
    for lo, hi in ((0, 4), (4, 8), (8, 16), (16, 24), (24, 48), (0, 48)):
        m = (rho >= lo) & (rho < hi)
        a, o = a_scat[m].sum(), o_scat[m].sum()
        c = a * n / 57.0                                   # scattered photons, about 57 keV each
        assert o == pytest.approx(a, rel=4.0 * math.sqrt(2.0 / c) + 0.002), (lo, hi, o, a, c)
