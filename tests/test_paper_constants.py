"""The library's defaults against the hyperparameters the paper prints (Supp. A), kept as
a cited fixture in tests/golden/paper_constants.json."""
import json
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_constants.json")


@pytest.fixture(scope="module")
def paper():
    with open(GOLDEN) as f:
        return json.load(f)


def test_mapping_learning_rates(paper):
    from paper_2603_21055_gb300 import mapping
    assert mapping.LR == paper["mapping_learning_rates"]


def test_eq1_weights(paper):
    from paper_2603_21055_gb300 import learned, parallel
    w = paper["eq1_loss_weights"]
    assert parallel.WEIGHTS == dict(rgb=w["rho"], ssim=w["tau"], depth=w["sigma"])
    assert (learned.RGB_WEIGHT, learned.DEPTH_WEIGHT) == (w["rho"], w["sigma"])


def test_tracking_defaults_are_the_replica_setting(paper):
    from paper_2603_21055_gb300 import binding as B
    p = B.sgad_gicp_default_params()
    assert p.stride == paper["tracking_downsampling_ratio_R"]["replica"]
    assert p.k_cov == paper["tracking_neighbours_K_c"]["replica"]
    # every dataset's K_c is accepted by the library
    for k in paper["tracking_neighbours_K_c"].values():
        q = B.sgad_gicp_default_params()
        q.k_cov = k
        assert B.sgad_gicp_workspace_size(q) > 0


def test_sequence_mapping_iterations(paper):
    import inspect
    from paper_2603_21055_gb300 import parallel
    it = inspect.signature(parallel.FrameMapper.__init__).parameters["iters"].default
    assert it == paper["mapping_iterations"]["replica"]


def test_current_view_share(paper):
    """Supp. A: at least 40 % of a frame's mapping iterations go to the current view."""
    from paper_2603_21055_gb300 import parallel
    for nn in (0, 1, 2, 4):
        for iters in (100, 500, 7):
            own = sum(parallel.view_of_iteration(it, nn) == 0 for it in range(iters))
            assert own >= paper["current_view_min_share"] * iters, (nn, iters)
