"""The oracle's pins must catch plausible mistakes.  Each case compiles a copy
of the C oracle with one mistake planted (a flipped sign, a wrong exponent, an
off-by-one bin, a wrong rounding rule), points the oracle at it, and checks
that the pin meant to catch it fails.  CPU only."""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "srs_oracle.c")

MUTANTS = [
    # (name, original text, mistake, pins that must fail)
    ("spectrum sign", "im[b] -= x[j] * sin(ang);", "im[b] += x[j] * sin(ang);",
     ["test_tone_in_tau_gives_exactly_n", "test_uniform_limit_is_the_fft", "test_tiny_spectra_against_brute_force"]),
    ("resampled-time exponent", "(-expm1((5.0 / 8.0) * log1p(-x)))", "(-expm1((3.0 / 8.0) * log1p(-x)))",
     ["test_delta_matches_high_precision_eq_new_t", "test_tone_in_tau_gives_exactly_n",
      "test_delta_derivative_is_frequency_ratio", "test_tiny_spectra_against_brute_force"]),
    ("bin frequency off by one", "double fb = f_lo + (double)b / t_coh;", "double fb = f_lo + (double)(b + 1) / t_coh;",
     ["test_uniform_limit_is_the_fft", "test_noiseless_exact_template_chirp_concentrates_power",
      "test_tiny_spectra_against_brute_force"]),
    ("beta frequency power", "pow(f0, 8.0 / 3.0);\n}", "pow(f0, 5.0 / 3.0);\n}",
     ["test_beta_range_matches_paper", "test_band_crossing_times_match_paper"]),
    ("whole-segment rounding", "double k = floor(t / t_coh);", "double k = ceil(t / t_coh);",
     ["test_injection_segment_count_matches_paper"]),
    ("duration exponent", "(1.0 - pow(f0 / f_end, 8.0 / 3.0))", "(1.0 - pow(f0 / f_end, 5.0 / 3.0))",
     ["test_injection_segment_count_matches_paper", "test_frequency_reaches_f_end_after_duration"]),
    ("segment start one segment late", "double t_i0 = J->local ? 0.0 : (double)i * (double)J->n_s / J->fs;",
     "double t_i0 = J->local ? 0.0 : (double)(i + 1) * (double)J->n_s / J->fs;",
     ["test_tiny_spectra_against_brute_force"]),
    ("local map referenced to the data start", "double t_i0 = J->local ? 0.0 : (double)i * (double)J->n_s / J->fs;",
     "double t_i0 = (double)i * (double)J->n_s / J->fs;",
     ["test_tiny_spectra_against_brute_force"]),
    ("literal resampled-time exponent", "pow(1.0 - (8.0 / 3.0) * beta * t, 5.0 / 8.0) / beta;",
     "pow(1.0 - (8.0 / 3.0) * beta * t, 3.0 / 8.0) / beta;",
     ["test_tau_literal_matches_high_precision_eq_new_t", "test_tau_derivative_is_frequency_ratio",
      "test_tau_difference_is_the_segment_local_delta"]),
    ("literal resampled time without 1/beta", "pow(1.0 - (8.0 / 3.0) * beta * t, 5.0 / 8.0) / beta;",
     "pow(1.0 - (8.0 / 3.0) * beta * t, 5.0 / 8.0);",
     ["test_tau_derivative_is_frequency_ratio"]),
]


@pytest.mark.parametrize("name,orig,bad,catchers", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, monkeypatch, name, orig, bad, catchers):
    src = open(SRC).read()
    assert src.count(orig) == 1, name
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(orig, bad))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(mutant), "-lm", "-lpthread"])
    monkeypatch.setattr(oracle, "_LIB", oracle.load(str(so)))
    for pin in catchers:
        fn = getattr(pins, pin)
        with pytest.raises(AssertionError):
            fn()


def test_pins_pass_on_the_unmodified_oracle(tmp_path, monkeypatch):
    so = tmp_path / "libsame.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), SRC, "-lm", "-lpthread"])
    monkeypatch.setattr(oracle, "_LIB", oracle.load(str(so)))
    for _, _, _, catchers in MUTANTS:
        for pin in catchers:
            getattr(pins, pin)()


# Mistakes planted in the numpy half of the oracle (power, segment sum,
# n_sigma), caught by the semicoherent pins.
SUM_MUTANTS = [
    ("one segment short", "for i in range(int(nsegs[m]))]", "for i in range(int(nsegs[m]) - 1)]",
     ["test_semicoherent_exact_chirp_closed_form", "test_semicoherent_against_per_item_brute_force"]),
    ("powers summed into the wrong row", "S[m] += P[k]", "S[0] += P[k]",
     ["test_semicoherent_exact_chirp_closed_form", "test_semicoherent_against_per_item_brute_force"]),
    ("segments counted from the second", "items = [(m, i) for m in range(len(betas)) for i in range(int(nsegs[m]))]",
     "items = [(m, i + 1) for m in range(len(betas)) for i in range(int(nsegs[m]))]",
     ["test_semicoherent_against_per_item_brute_force"]),
    ("n_sigma divided by N", "(S - 2.0 * nseg_) / (2.0 * np.sqrt(nseg_))", "(S - 2.0 * nseg_) / (2.0 * nseg_)",
     ["test_semicoherent_exact_chirp_closed_form", "test_semicoherent_against_per_item_brute_force"]),
    ("power without its factor 2", "return 2.0 * np.abs(F) ** 2 / n_s", "return np.abs(F) ** 2 / n_s",
     ["test_semicoherent_exact_chirp_closed_form", "test_semicoherent_against_per_item_brute_force"]),
]


@pytest.mark.parametrize("name,orig,bad,catchers", SUM_MUTANTS, ids=[m[0] for m in SUM_MUTANTS])
def test_sum_pins_catch_planted_mistake(monkeypatch, name, orig, bad, catchers):
    import types
    src = open(oracle.__file__).read()
    assert src.count(orig) == 1, name
    mod = types.ModuleType("oracle_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(orig, bad), "oracle_mutant.py", "exec"), mod.__dict__)
    for fn in ("power", "n_sigma", "semicoherent"):
        monkeypatch.setattr(oracle, fn, getattr(mod, fn))
    for pin in catchers:
        with pytest.raises(AssertionError):
            getattr(pins, pin)()


def test_power_normalisation_pin(monkeypatch):
    """P = 2|F|^2/n_s (Sec. III.C); dropping the factor 2 breaks the noise pin."""
    monkeypatch.setattr(oracle, "power", lambda F, n_s: abs(F) ** 2 / n_s)
    with pytest.raises(AssertionError):
        pins.test_noise_power_moments_and_n_sigma_null()


# Mistakes planted in the two-stage oracle (oracle/slide.py), caught by the
# pins in test_oracle_slide.py.
SLIDE_MUTANTS = [
    ("t0 fraction sign", "off = (1.0 if c > 0 else 0.0) - c", "off = (1.0 if c > 0 else 0.0) + c",
     ["test_track_frequency_is_the_phase_derivative", "test_track_length_matches_band_time"]),
    ("bin rounded down", "j = int(np.rint((f - f_lo) * t_coh))", "j = int(np.floor((f - f_lo) * t_coh))",
     ["test_track_frequency_is_the_phase_derivative"]),
    ("bank entry for beta at f0", "bl = beta(mc, f)", "bl = beta(mc, f0)",
     ["test_track_bank_index_is_nearest_local_beta"]),
    ("power not centred", "np.sum((P_track - 2.0) / 2.0)", "np.sum(P_track / 2.0)",
     ["test_stack_slide_closed_forms"]),
    ("segment containing t0 kept", "return n + (1 if c > 0 else 0)", "return n",
     ["test_stack_slide_brute_force_on_a_random_cube"]),
    ("local map referenced to t = 0", "items, n_threads=n_threads, local=True)", "items, n_threads=n_threads, local=False)",
     ["test_power_cube_concentrates_an_entering_chirp"]),
    ("amplitude to the power 2/3", "(f / f0) ** (4.0 / 3.0)", "(f / f0) ** (2.0 / 3.0)",
     ["test_amplitude_average_matches_closed_form"]),
    ("weights not normalised", "/ np.sqrt(np.sum(a * a)))\n\n\ndef whiten", ")\n\n\ndef whiten",
     ["test_weighted_stack_slide_closed_forms"]),
    ("power not divided by the PSD", "a * (P / S - 2.0) / 2.0", "a * (P - 2.0) / 2.0",
     ["test_weighted_stack_slide_closed_forms"]),
    ("whitening without the segment deviation", "return 2.0 + 2.0 * (Pt - mu) / sigma, S, mu, sigma",
     "return 2.0 + 2.0 * (Pt - mu), S, mu, sigma", ["test_whitening_moments_and_psd_estimate"]),
    ("PSD estimate without the factor 2", "S = P.mean(axis=2) / 2.0 if s_eff is None", "S = P.mean(axis=2) if s_eff is None",
     ["test_whitening_moments_and_psd_estimate"]),
]


@pytest.mark.parametrize("name,orig,bad,catchers", SLIDE_MUTANTS, ids=[m[0] for m in SLIDE_MUTANTS])
def test_slide_pins_catch_planted_mistake(monkeypatch, name, orig, bad, catchers):
    import types
    import test_oracle_slide as spins
    from oracle import slide
    src = open(slide.__file__).read()
    assert src.count(orig) == 1, name
    mod = types.ModuleType("oracle.slide_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(orig, bad), "slide_mutant.py", "exec"), mod.__dict__)
    for fn in ("local_bank", "power_cube", "first_segment", "track", "n_sigma_track", "stack_slide", "amplitude_sq",
               "n_sigma_weighted", "whiten"):
        monkeypatch.setattr(slide, fn, getattr(mod, fn))
    for pin in catchers:
        fn = getattr(spins, pin)
        args = {"test_track_frequency_is_the_phase_derivative": [(6e-2, 0.25), (1e-2, 0.0)],
                "test_track_length_matches_band_time": [(1e-1, 0.5)],
                "test_amplitude_average_matches_closed_form": [(1e-1, 0.6, 34)]}.get(pin)
        with pytest.raises(AssertionError):
            if args:
                for a in args:
                    fn(*a)
            else:
                fn()


# Mistakes planted in the statistics oracle (oracle/stats.py), caught by the
# oracle pins of test_stats.py.
STATS_MUTANTS = [
    ("chi-square with 2N - 1 dof", "return brentq(lambda lam: ncx2.sf(s, 2 * n_seg, lam) - p_det",
     "return brentq(lambda lam: ncx2.sf(s, 2 * n_seg - 1, lam) - p_det",
     ["test_oracle_detection_noncentrality_matches_paper"]),
    ("threshold not centred", "return (s - 2.0 * n_seg) / (2.0 * np.sqrt(n_seg))", "return s / (2.0 * np.sqrt(n_seg))",
     ["test_oracle_one_segment_threshold_closed_form"]),
    ("hypoexponential coefficient inverted", "c *= wi / (wi - wj)", "c *= wj / (wi - wj)",
     ["test_oracle_weighted_law_monte_carlo"]),
    ("characteristic function's factor 2", "z = 1.0 - 2.0j * w * t", "z = 1.0 - 1.0j * w * t",
     ["test_oracle_weighted_noncentral_law_reduces_to_textbook_laws"]),
    ("signal term without its weight", "np.exp(1j * lam * w * t / z)", "np.exp(1j * lam * t / z)",
     ["test_oracle_detection_probability_monte_carlo"]),
    ("inversion with the wrong sign", "return 0.5 + (head + c - s) / np.pi", "return 0.5 - (head + c - s) / np.pi",
     ["test_oracle_weighted_noncentral_law_reduces_to_textbook_laws"]),
]


@pytest.mark.filterwarnings("ignore::RuntimeWarning")     # a planted mistake may give a probability outside [0, 1]
@pytest.mark.parametrize("name,orig,bad,catchers", STATS_MUTANTS, ids=[m[0] for m in STATS_MUTANTS])
def test_stats_pins_catch_planted_mistake(monkeypatch, name, orig, bad, catchers):
    import types
    import test_stats as spins
    from oracle import stats
    src = open(stats.__file__).read()
    assert src.count(orig) == 1, name
    mod = types.ModuleType("oracle.stats_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(orig, bad), "stats_mutant.py", "exec"), mod.__dict__)
    for fn in ("nsigma_threshold_equal", "detection_noncentrality", "weighted_exp_sf", "nsigma_threshold_weighted",
               "detection_probability_mc", "weighted_noncentral_sf", "detection_probability"):
        monkeypatch.setattr(stats, fn, getattr(mod, fn))
    for pin in catchers:
        with pytest.raises(Exception):
            getattr(spins, pin)()
