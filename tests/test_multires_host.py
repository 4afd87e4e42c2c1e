"""Host-side rule of the multi-resolution stack: the layer count
(sg_multires_layers, no GPU needed) and the layer specs."""
import pytest

import sg_inputs as si

sg = pytest.importorskip("paper_2512_11473_b300")


def _brute(dims, min_dims):
    L, d = 1, list(dims)
    while all(v % 2 == 0 and v // 2 >= min_dims for v in d):
        d = [v // 2 for v in d]
        L += 1
    return L


@pytest.mark.parametrize("dims,min_dims,want", [((256, 256, 256), 8, 6), ((256, 256, 256), 16, 5),
                                                ((250, 250, 100), 8, 2), ((175, 150, 175), 8, 1),
                                                ((64, 32, 16), 4, 3), ((8, 8, 8), 8, 1), ((16, 16, 16), 1, 5)])
def test_layer_count(dims, min_dims, want):
    spec = si.GridSpec((0.0, 0.0, 0.0), dims, 0.01)
    assert sg.multires_layers(spec, min_dims) == want == _brute(dims, min_dims)


def test_layer_specs_cover_the_domain():
    spec = si.shelled_sphere()[1]
    L = sg.multires_layers(spec)
    for k in range(L):
        s = sg.layer_spec(spec, k, L)
        assert s.lo == spec.lo
        assert s.h == spec.h * 2 ** (L - 1 - k)
        for a in range(3):
            assert s.dims[a] * s.lc == pytest.approx(spec.dims[a] * spec.lc)
    assert sg.layer_spec(spec, L - 1, L) == spec
