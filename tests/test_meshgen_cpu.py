"""Host checks of the seeded input generators (no method arithmetic).

The unstructured Delaunay boxes must be valid conforming tetrahedrisations of
the box: positive volumes summing to the box volume, every interior face
shared by exactly two cells, every boundary face on the box surface; the
boundary-face extractor must find exactly the box surface.
"""
import numpy as np
import pytest

from paper_1804_10060_gb300 import meshgen


@pytest.mark.parametrize("hub", [0, 60])
def test_delaunay_box_is_a_conforming_tetrahedrisation(hub):
    coords, cells, q = meshgen.delaunay_box(6, seed=3, hub=hub)
    x = coords[cells]
    vol = np.einsum("ij,ij->i", np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), x[:, 3] - x[:, 0]) / 6.0
    assert vol.min() > 0 and q["min_volume"] == pytest.approx(vol.min())
    assert vol.sum() == pytest.approx(2.0, rel=1e-12)
    faces = np.sort(np.concatenate([cells[:, list(f)] for f in meshgen.TET_FACES]), axis=1)
    _, counts = np.unique(faces, axis=0, return_counts=True)
    assert counts.max() == 2
    bf = meshgen.boundary_faces(cells)
    fx = coords[bf]
    on_surface = np.zeros(len(bf), bool)
    for d, L in enumerate((2.0, 1.0, 1.0)):
        on_surface |= np.all(np.abs(fx[:, :, d]) < 1e-12, axis=1) | np.all(np.abs(fx[:, :, d] - L) < 1e-12, axis=1)
    assert on_surface.all()
    area = 0.5 * np.linalg.norm(np.cross(fx[:, 1] - fx[:, 0], fx[:, 2] - fx[:, 0]), axis=1).sum()
    assert area == pytest.approx(2 * (2 + 2 + 1), rel=1e-12)
    if hub:
        assert q["max_valence"] >= 2 * hub - 20
    assert q["min_dihedral_deg"] > 0


def test_boundary_faces_of_p2_cube():
    pb = meshgen.unit_cube_problem(3, 2)
    f = meshgen.boundary_faces(pb.cells)
    assert f.shape == (6 * 9 * 2, 6)
    # the mid-edge nodes sit at the midpoints of the face's edges
    for k, (a, b) in enumerate(((0, 1), (1, 2), (2, 0))):
        mid = 0.5 * (pb.coords[f[:, a]] + pb.coords[f[:, b]])
        assert np.abs(pb.coords[f[:, 3 + k]] - mid).max() < 1e-14
