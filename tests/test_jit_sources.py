"""The shape-specialised stage kernels compile at run time (NVRTC) from the
device headers embedded in the library.  NVRTC needs no device, so every
model, dimension and scheme is compiled here on the CPU; on the GPU the
parity tests run the compiled kernels themselves."""
import pytest

from paper_2101_05916_gb300 import hj

CASES = ([("quad_x4", [41, 41, 41, 41], s, t) for s in (1, 2, 5) for t in (128, 256, 512)]
         + [("quad_z", [1025, 1025], s, t) for s in (1, 2, 5) for t in (128, 256, 512)]
         + [("drift", n, s, 256) for n in ([1 << 20], [1025, 1025], [101, 103, 107],
                                            [33, 35, 37, 39]) for s in (1, 2, 5)])


@pytest.mark.parametrize("model,n,scheme,threads", CASES,
                         ids=["%s-%dd-s%d-t%d" % (m, len(n), s, t) for m, n, s, t in CASES])
def test_specialised_source_compiles(model, n, scheme, threads):
    hj.hj_jit_check(n, model, scheme, threads)


def test_bad_arguments_are_rejected():
    with pytest.raises(hj.HJError):
        hj.hj_jit_check([41] * 4, "quad_x4", 3, 256)
    with pytest.raises(hj.HJError):
        hj.hj_jit_check([41] * 4, "quad_x4", 5, 300)
    with pytest.raises(hj.HJError):
        hj.hj_jit_check([2, 41], "quad_z", 2, 256)


def test_large_grid_stage_kernels_fit_2048_threads_per_sm_without_spills():
    """The WENO5 stage kernels of the x-subsystem (box on the position axis)
    compiled for 81^4 and 61^4 grids run 2048 resident threads per SM: 32
    registers per thread, nothing spilled.  41^4 keeps 1536 threads (40
    registers), also without spills."""
    for n in (81, 61):
        for threads in (128, 256, 512):
            regs, spill = hj.hj_jit_check_resources([n] * 4, "quad_x4", 5, threads)
            assert regs <= 32 and spill == 0, (n, threads, regs, spill)
    regs, spill = hj.hj_jit_check_resources([41] * 4, "quad_x4", 5, 256)
    assert 32 < regs <= 40 and spill == 0, (regs, spill)
    regs, spill = hj.hj_jit_check_resources([1025, 1025], "quad_z", 2, 256, con_axes=(0, 1))
    assert regs <= 40 and spill == 0
    for bad in ((), (4,)):
        with pytest.raises(hj.HJError):
            hj.hj_jit_check_resources([81] * 4, "quad_x4", 5, 256, con_axes=bad)


TILE_CASES = ([("quad_x4", [41, 41, 41, 41], s, r) for s in (1, 2, 5) for r in (3, 6, 7)]
              + [("quad_x4", [81, 81, 81, 81], 5, r) for r in (3, 5, 12)]
              + [("quad_z", [201, 201], s, r) for s in (2, 5) for r in (1, 2, 5)]
              + [("drift", n, 5, 2) for n in ([300, 5], [101, 103], [33, 35, 37], [9, 11, 13, 15])])


@pytest.mark.parametrize("model,n,scheme,rows", TILE_CASES,
                         ids=["%s-%dd-s%d-r%d" % (m, len(n), s, r) for m, n, s, r in TILE_CASES])
def test_specialised_row_tile_source_compiles(model, n, scheme, rows):
    hj.hj_jit_check_tiles(n, model, scheme, rows)


def test_row_tiles_that_do_not_fit_are_rejected():
    with pytest.raises(hj.HJError):
        hj.hj_jit_check_tiles([81] * 4, "quad_x4", 5, 13)  # 1053 nodes > 1024
    with pytest.raises(hj.HJError):
        hj.hj_jit_check_tiles([300], "drift", 5, 2)  # one line only
    with pytest.raises(hj.HJError):
        hj.hj_jit_check_tiles([41] * 4, "quad_x4", 5, 0)


GROUPS = [
    [((61, 61, 61, 61), "quad_x4", 5), ((61, 61, 61, 61), "quad_x4", 5), ((201, 201), "quad_z", 2)],
    [((31, 31, 31, 31), "quad_x4", 5), ((101, 101), "quad_z", 2), ((401, 401), "quad_z", 2)],
    [((13, 15, 9, 19), "drift", 2), ((300,), "drift", 5), ((40, 31), "drift", 1)],
]


@pytest.mark.parametrize("grids", GROUPS, ids=["decomposed", "serving-mix", "drift-mix"])
def test_group_kernel_source_compiles(grids):
    hj.hj_jit_check_group(grids)


def test_group_kernel_bad_arguments_are_rejected():
    with pytest.raises(hj.HJError):
        hj.hj_jit_check_group([((41, 41), "quad_x4", 5)])  # no such stencil
    with pytest.raises(hj.HJError):
        hj.hj_jit_check_group([((41, 2), "drift", 2)])  # an axis with fewer than 3 nodes
    with pytest.raises(hj.HJError):
        hj.hj_jit_check_group([((41, 41), "quad_z", 3)])  # no such scheme
