"""B300-native periodic lattice homogenization: a matrix-free geometric-multigrid V-cycle
on a sparse active-voxel hierarchy, behind the C ABI of include/gmt.h (libgmt.so).

    from paper_2604_26518_b300 import gmt
    h = gmt.Hierarchy(voxels)                      # N^3 uint8, N a multiple of 4
    status, u, info = h.solve(gmt.ELASTIC, E=1.0, nu=0.3, tol=1e-5)
    CH = h.homogenize(gmt.ELASTIC, E=1.0, nu=0.3)  # 6 x 6

`lattices` holds the seeded synthetic cell generators (inputs only).
"""
