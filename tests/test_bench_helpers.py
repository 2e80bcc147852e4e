"""Host helpers of bench.py: the Gauss-point count behind the adjoint's byte accounting against the
oracle's face list, on meshes with every cell type, periodic pairs and boundaries."""
import meshgen as mg


def test_gauss_point_count_matches_the_oracle(orc):
    import bench
    for mesh in (mg.ramp_box(8, 4, 2, n_prism=1), mg.periodic_box(6), mg.pyramid_box(6, periodic=False),
                 mg.wall_box(6, 4, 8, n_prism=3)):
        F = orc.Mesh(mesh).faces()
        assert bench.mg_gauss_points(mesh) == int(F["ngp"].sum())
