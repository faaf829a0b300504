"""Host-side argument checks of the application bindings, which run before
any device memory is touched."""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_1809_07444_gb300.apps import Sugarscape, Traffic  # noqa: E402


def test_sugarscape_rejects_two_agents_on_one_cell():
    cap = np.zeros((20, 20), np.uint8)
    a = np.array([[3, 4, 10, 1, 2, 0, 80], [3, 4, 12, 2, 3, 0, 90]], np.int32)
    with pytest.raises(ValueError, match="one cell"):
        Sugarscape(20, 20, cap, a, 1)


@pytest.mark.parametrize("xy", [(-1, 0), (20, 3), (5, 20), (5, -2)])
def test_sugarscape_rejects_agents_off_the_torus(xy):
    cap = np.zeros((20, 20), np.uint8)
    a = np.array([[xy[0], xy[1], 10, 1, 2, 0, 80]], np.int32)
    with pytest.raises(ValueError, match="outside"):
        Sugarscape(20, 20, cap, a, 1)


def test_sugarscape_rejects_a_landscape_of_the_wrong_size():
    with pytest.raises(ValueError, match="W \\* H"):
        Sugarscape(20, 20, np.zeros((19, 20), np.uint8), np.zeros((0, 7), np.int32), 1)


def test_traffic_rejects_a_start_of_the_wrong_size():
    with pytest.raises(ValueError, match="R \\* L"):
        Traffic(4, 100, np.full((4, 99), -1, np.int8), 1)
