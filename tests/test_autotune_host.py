"""Host side of the autotuner: the tuning file it writes and reads (the
format ahf_create applies), the device key, and the search's knob list."""
import os

import pytest

from paper_0904_3662_gb300 import ahf, autotune


def test_device_key_matches_the_library_rule():
    assert autotune.device_key("NVIDIA GB300") == "NVIDIA_GB300"
    assert autotune.device_key("a/b c-1.0_x") == "a_b_c-1.0_x"


def test_tuning_file_round_trip(tmp_path):
    p = str(tmp_path / "t.txt")
    opts = {ahf.OPT_PROMOTE: 0, ahf.OPT_CLASS_CUT + 2: 3072, ahf.OPT_PASS_CHUNK: 16}
    autotune.write(p, "NVIDIA_GB300", "0123456789abcdef", opts, "batch\ndefault 1 ms, tuned 0.9 ms")
    t = autotune.read(p)
    assert t["device"] == "NVIDIA_GB300" and t["build"] == "0123456789abcdef"
    assert t["options"] == opts
    assert t["comment"] == ["batch", "default 1 ms, tuned 0.9 ms"]
    assert autotune.valid_for(p, "NVIDIA_GB300", "0123456789abcdef")
    assert not autotune.valid_for(p, "NVIDIA_GB300", "fedcba9876543210")
    assert not autotune.valid_for(p, "OTHER", "0123456789abcdef")
    assert not autotune.valid_for(str(tmp_path / "missing.txt"), "NVIDIA_GB300", "0123456789abcdef")
    with open(p, "a") as f:
        f.write("bogus line\n")
    with pytest.raises(ValueError):
        autotune.read(p)


def test_knobs_start_at_the_library_defaults():
    ks = autotune.knobs(ahf, multi_cta=True)
    opts = [o for o, _ in ks]
    assert opts[0] == ahf.OPT_PROMOTE and ks[0][1][0] == 1
    for v, cap in enumerate(ahf.VARIANT_CAPS[:-1]):
        vals = dict(ks)[ahf.OPT_CLASS_CUT + v]
        assert vals[0] == cap and all(0 < x <= cap for x in vals)
    assert dict(ks)[ahf.OPT_PASS_CHUNK][0] == 8
    assert ahf.OPT_PASS_CHUNK not in [o for o, _ in autotune.knobs(ahf, multi_cta=False)]


def test_build_id_is_the_source_hash():
    from paper_0904_3662_gb300 import build_lib
    build_lib.build()
    assert ahf.build_id() == build_lib.source_hash()
