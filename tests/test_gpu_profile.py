"""Profiling modes: serial lanes add up launch by launch; concurrent lanes
report each kernel class's active wall time, never more than the sum of its
launches."""
import pytest

from paper_2202_13511_gb300 import mpdp
from paper_2202_13511_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_profile_modes():
    qs = [W.snowflake(16, seed=i) for i in range(8)] + [W.cyclic(14, seed=i) for i in range(4)]
    with mpdp.Optimizer(0) as o:
        o.set_config(lanes=4)
        want = [p.cost for p in o.optimize_batch(qs)]
        got = {}
        for mode in (mpdp.PROFILE_SERIAL, mpdp.PROFILE_CONCURRENT):
            o.profile(mode)
            assert [p.cost for p in o.optimize_batch(qs)] == want
            got[mode] = o.profile_read()
            o.profile(mpdp.PROFILE_OFF)
        s, c = got[mpdp.PROFILE_SERIAL], got[mpdp.PROFILE_CONCURRENT]
        # per lane one filter launch per kind present: the connected-set
        # unranking for the trees, the bitmap sweep for the cyclic queries
        assert 4 <= s["filter"]["launches"] <= 8
        for k in s:
            assert s[k]["launches"] == c[k]["launches"]
            assert s[k]["active_ms"] == pytest.approx(s[k]["ms"], rel=1e-3, abs=1e-3)
            assert c[k]["active_ms"] <= c[k]["ms"] * (1 + 1e-6) + 1e-6
        for bad in (3, -1):
            with pytest.raises(mpdp.MPDPError) as ei:
                o.profile(bad)
            assert ei.value.code == mpdp.ERR["INVALID_ARG"]
