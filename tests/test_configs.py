"""The JSON scene configurations (CPU): each file in the package's configs/
holds the scene parameters and depth intrinsics of the synthetic workload of
the same name, and the loader refuses files with unknown or missing fields."""

import json

import pytest

import paper_1708_00783_gb300 as itm
from synth import workload_by_name


@pytest.mark.parametrize("name", ["tiny", "kinect", "large"])
def test_config_matches_the_workload(name):
    params, intr = itm.load_config(name)
    w = workload_by_name(name, n_frames=2)
    assert params == dict(w.params, weight_mode=0)
    i = w.intr
    assert (intr.width, intr.height, intr.fx, intr.fy, intr.cx, intr.cy) == (i.width, i.height, i.fx, i.fy, i.cx,
                                                                                i.cy)
    itm.make_params(**params)  # every field is a scene parameter


def test_config_from_a_path_and_bad_fields(tmp_path):
    params, _ = itm.load_config("tiny")
    good = {"scene": params, "intrinsics": {"width": 8, "height": 6, "fx": 5.0, "fy": 5.0, "cx": 3.5, "cy": 2.5}}
    p = tmp_path / "c.json"
    p.write_text(json.dumps(good))
    got, intr = itm.load_config(str(p))
    assert got == params and intr.width == 8
    for bad in ({"scene": dict(params, voxels=1), "intrinsics": good["intrinsics"]},
                {"scene": {k: v for k, v in params.items() if k != "mu"}, "intrinsics": good["intrinsics"]},
                {"scene": params, "intrinsics": {"width": 8}}):
        p.write_text(json.dumps(bad))
        with pytest.raises(ValueError):
            itm.load_config(str(p))
