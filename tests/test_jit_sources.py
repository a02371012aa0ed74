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
