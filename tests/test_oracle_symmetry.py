"""k-point symmetry by the small group of Q (Sec. 2.6), pinned against the full k-mesh.

The oracle run on the irreducible wedge of the small group of Q (k-point weights = star
sizes, the response density averaged over the group) must give the Lanczos coefficients of
the run on the whole mesh: every quantity the recursions form is a sum over the mesh, and
the terms of a star are the rotated terms of its representative.  The small group itself is
checked against its definition (a group; R Q = Q; R maps the crystal onto itself), and a
planted mistake (the average over the group left out) must break the agreement.
"""
import copy

import numpy as np
import pytest

import workloads as w
from oracle import lanczos
from oracle.liouvillian import System
from workloads.cells import irreducible_kpoints, kmesh_frac, small_group


def test_small_group_of_q_along_x():
    spec = w.config_small(True)
    ops = small_group(spec)
    assert len(ops) == 4                                  # C2v: E, C2 about x, two mirrors through x
    assert np.allclose(ops[0], np.eye(3))
    for r in ops:
        assert np.allclose(r @ spec.q_cart, spec.q_cart)
        assert np.allclose(r @ r.T, np.eye(3))
        for s in ops:                                     # closed under products
            assert any(np.allclose(r @ s, t) for t in ops)
    generic = w.config_small(True)
    generic.q_cart = np.array([0.031, 0.017, 0.007])
    assert len(small_group(generic)) == 1


def test_irreducible_kpoints_cover_the_mesh_once():
    spec = w.config_kb(True)
    ops = small_group(spec)
    kf, mult = irreducible_kpoints(spec, ops)
    n = np.array(spec.kmesh)
    assert mult.sum() == np.prod(n)
    images = {}
    for i, f in enumerate(kf):
        star = {tuple(np.round(((r @ (f @ spec.bvec)) @ np.linalg.inv(spec.bvec)) * n).astype(int) % n) for r in ops}
        assert len(star) == mult[i]
        for s in star:
            assert s not in images
            images[s] = i
    assert set(images) == {tuple(np.round(f * n).astype(int) % n) for f in kmesh_frac(spec.kmesh)}


@pytest.fixture(scope="module")
def pair():
    return w.get_bundle(w.config_small()), w.get_bundle(w.config_small(True))


@pytest.mark.parametrize("flavour,steps", [("ph", 60), ("nh", 40)])
def test_irreducible_wedge_gives_full_mesh_coefficients(pair, flavour, steps):
    full, ibz = pair
    assert ibz.nks < full.nks
    a = lanczos.run(System(full), steps, flavour)
    b = lanczos.run(System(ibz), steps, flavour)
    assert np.max(np.abs(a.beta - b.beta) / np.abs(a.beta)) < 1e-12
    assert np.max(np.abs(a.gamma - b.gamma) / np.abs(a.gamma)) < 1e-12
    assert np.max(np.abs(a.z - b.z)) / np.max(np.abs(a.z)) < 1e-12


def test_planted_mistake_without_the_group_average(pair):
    full, ibz = pair
    broken = copy.copy(ibz)
    broken.sym = None                                     # weights kept, density not averaged
    a = lanczos.run(System(full), 20, "ph")
    b = lanczos.run(System(broken), 20, "ph")
    assert np.max(np.abs(a.beta - b.beta) / np.abs(a.beta)) > 1e-6
