"""Full-band search driver on a narrow band: recovered sources sit on injected
ones and every recovery gets a valid posterior round."""
import pytest

from paper_2307_03763_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2307_03763_gb300 import api, build
    build.build()
    return api


def test_fullband_narrow_band(api):
    # 400 binaries over 2-2.6 mHz (416 windows): by chance a recovery would sit
    # within a bin of an injected source about 2% of the time.  Scored by the
    # paper's match metrics (Sec. IV): measured 67% of recoveries with
    # delta < 0.3 and 68% with overlap > 0.9, 207 of the 354 injections above
    # SNR 10 matched (Gaussian posteriors, all windows at once; 64%, 65% and
    # 225 with the even/odd runs on median-noise weights), with f0 searched
    # over the padded segment and signals found in the padding subtracted but
    # not catalogued (Alg. 2)
    from paper_2307_03763_gb300 import fullband
    ctx = api.Context(2 * wk.YEAR)
    for post, scheme, noise in (("gauss", "all", "true"), ("kde", "all", "true"), ("gauss", "evenodd", "median")):
        st = fullband.run(ctx, n_src=400, f_lo=2e-3, f_hi=2.6e-3, rounds=2, pop=1024, generations=200, n_post=2000,
                          posterior=post, warm=post == "gauss" and scheme == "all", scheme=scheme, noise=noise,
                          amp="loguniform")
        assert st["windows"] == len(wk.fullband_layout(2e-3, 2.6e-3, 2 * wk.YEAR))
        assert st["recovered"] > 100, st
        assert st["within_1_bin"] >= 0.5 and st["within_3_bins"] >= 0.7, st
        assert st["posteriors"] == st["recovered"]
        assert st["median_accept_rate"] > 0.0, st
        key = {k: st.get(k) for k in ("recovered", "median_accept_rate", "delta_lt_0.3", "overlap_gt_0.9",
                                      "matched_injected_delta_lt_0.3", "windows_with_several_sources")}
        assert st["delta_lt_0.3"] >= 0.5 and st["overlap_gt_0.9"] >= 0.5, key
        assert st["matched_injected_delta_lt_0.3"] >= 170, key
        assert st["padding_signals_subtracted"] > 100, key
        if post == "gauss" and scheme == "all":
            # posteriors at the joint estimates on d minus every other found
            # signal: measured 22% median acceptance (16% without the joint refit)
            assert st["median_accept_rate"] >= 0.18, key
            assert st["windows_with_several_sources"] > 50 and st["joint_snr_median"] > 10.0, st
