"""Planted mistakes: each plausible slip in the oracle must fail some pin.

Every mutant below rewrites one expression of the oracle's source (a dropped
term, a flipped sign, a transposed operand, an off-by-one index, a
non-strict comparison, a missing step) and re-runs a set of pins against the
mutated module; at least one pin has to fail.  The mutation happens on the
CPU, in a private copy of the oracle module.
"""
import inspect
import sys
import types

import pytest

import oracle.ahf_oracle as real
from tests import test_oracle_pins as pins

MUTANTS = [
    # (name, function, original snippet, mutated snippet)
    ("inclusive_mass", "potential_sorted",
     "m_inner = np.concatenate([[0.0], np.cumsum(m)[:-1]])", "m_inner = np.cumsum(m)"),
    ("dropped_self_term", "potential_sorted",
     "outer = np.cumsum(mr[::-1])[::-1]", "outer = np.concatenate([np.cumsum(mr[::-1])[::-1][1:], [0.0]])"),
    ("wrong_sign_outer", "potential_sorted",
     "return -G * (inner + outer)", "return -G * (inner - outer)"),
    ("transposed_inner", "potential_sorted",
     "inner = np.where(rr > 0.0, m_inner / rr, 0.0)", "inner = np.where(rr > 0.0, m_inner * rr, 0.0)"),
    ("prefix_from_outside", "potential_sorted",
     "outer = np.cumsum(mr[::-1])[::-1]", "outer = np.cumsum(mr)"),
    ("non_strict_test", "unbind_halo", "unbound = u2 > two_phi", "unbound = u2 >= two_phi"),
    ("hubble_sign", "unbind_halo", "+ params.H * d[order]", "- params.H * d[order]"),
    ("no_bulk_subtraction", "unbind_halo", "u = v[order] - vbulk[None, :]", "u = v[order]"),
    ("unweighted_bulk", "unbind_halo",
     "vbulk = (ma[:, None] * v[alive]).sum(axis=0) / ma.sum()", "vbulk = v[alive].mean(axis=0)"),
    ("unsorted_list", "unbind_halo", "order = alive[np.lexsort((alive, r[alive]))]\n        phi",
     "order = alive\n        phi"),
    ("single_pass", "unbind_halo", "if not unbound.any():", "if True:"),
    ("exclusive_virial_mass", "virial", "mk = np.cumsum(m)", "mk = np.cumsum(m) - m"),
    ("virial_same_radius", "virial", "r_next = np.concatenate([r[1:], [np.inf]])",
     "r_next = np.concatenate([r[:-1], [np.inf]])"),
    ("virial_square_root", "virial", "** (1.0 / 3.0)", "** (1.0 / 2.0)"),
    ("min_image_sign", "recentre", "d = np.where(d > half, d - box, d)", "d = np.where(d > half, d + box, d)"),
]

PINS = [
    pins.test_phi_hand_worked, pins.test_phi_matches_appendix_a_integral,
    pins.test_phi_monotone_and_outer_value, pins.test_radius_order_matters,
    pins.test_virial_identity_and_counting, pins.test_virial_uniform_sphere_closed_form,
    pins.test_single_particle, pins.test_strict_inequality_keeps_marginal_particle,
    pins.test_vbulk_is_mass_weighted, pins.test_galilean_invariance,
    pins.test_infall_cancelling_hubble_flow_stays_bound, pins.test_gather_sphere_and_minimum_image,
    pins.test_idempotent, pins.test_all_unbound_gives_empty,
]


def _mutant_module(func_name, old, new, monkeypatch):
    src = inspect.getsource(real)
    fsrc = inspect.getsource(getattr(real, func_name))
    assert old in fsrc, (func_name, old)
    src = src.replace(fsrc, fsrc.replace(old, new, 1))
    mod = types.ModuleType("ahf_oracle_mutant")
    monkeypatch.setitem(sys.modules, "ahf_oracle_mutant", mod)
    exec(compile(src, "<mutant>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name,func,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, func, old, new, monkeypatch):
    mod = _mutant_module(func, old, new, monkeypatch)
    monkeypatch.setattr(pins, "O", mod)
    failed = []
    for pin in PINS:
        try:
            pin()
        except Exception:           # assertion or numerical blow-up both count
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"


from tests import test_oracle_props as props_pins

PROPS_MUTANTS = [
    ("props_no_half_kinetic", "halo_properties", "K = 0.5 * float(", "K = 1.0 * float("),
    ("props_no_half_potential", "halo_properties", "U = 0.5 * float(", "U = float("),
    ("props_no_bulk", "halo_properties", "u = v - vbar[None, :] + params.H * d", "u = v + params.H * d"),
    ("props_cross_transposed", "halo_properties", "np.cross(d, u)", "np.cross(u, d)"),
    ("props_mass_power", "halo_properties", "M ** 2.5", "M ** 1.5"),
    ("props_exclusive_mass_vc", "halo_properties", "m_in = np.cumsum(m)", "m_in = np.cumsum(m) - m"),
    ("props_virial_off_by_one", "halo_properties", "n = d.shape[0] if k_vir < 0 else k_vir + 1",
     "n = d.shape[0] if k_vir < 0 else k_vir"),
    ("match_xi_unsquared", "match_catalogs", "x = count[b] ** 2 / (n1 * len(lists_b[b]))",
     "x = count[b] / (n1 * len(lists_b[b]))"),
    ("match_tie_to_higher", "match_catalogs", "if x > xi[a]:", "if x >= xi[a]:"),
]

PROPS_PINS = [props_pins.test_two_particle_worked_example, props_pins.test_solid_body_rotation,
              props_pins.test_uniform_sphere_energy_and_rotation_curve, props_pins.test_nfw_rotation_curve_peak,
              props_pins.test_invariances_and_virial_selection, props_pins.test_match_catalogs_cases]


@pytest.mark.parametrize("name,func,old,new", PROPS_MUTANTS, ids=[m[0] for m in PROPS_MUTANTS])
def test_properties_mutant_is_caught(name, func, old, new, monkeypatch):
    mod = _mutant_module(func, old, new, monkeypatch)
    monkeypatch.setattr(props_pins, "O", mod)
    failed = []
    for pin in PROPS_PINS:
        try:
            pin()
        except Exception:
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"


from tests import test_oracle_variants as variant_pins

RISE_MUTANTS = [
    ("rise_edge_next_shell", "rise_edge", "return b[smin]", "return b[smin] + 1"),
    ("rise_edge_inner_radius", "rise_edge", "float(r[hi]) ** 3 - float(r[lo]) ** 3",
     "float(r[hi]) ** 3 - float(r[lo - 1]) ** 3 * 0.0"),
    ("rise_edge_no_rise_test", "rise_edge", "if any(rho[s] > rho[smin] for s in rho if s > smin):", "if True:"),
    ("rise_edge_max_not_min", "rise_edge", "smin = min(rho, key=lambda s: (rho[s], s))",
     "smin = max(rho, key=lambda s: (rho[s], s))"),
    ("rise_edge_shell_mass", "rise_edge", "(mk[hi] - mk[lo]) / vol", "mk[hi] / vol"),
]

RISE_PINS = [variant_pins.test_rise_edge_truncates_at_the_density_minimum,
             variant_pins.test_rise_edge_leaves_other_haloes_alone, variant_pins.test_rise_edge_uses_shell_masses]


@pytest.mark.parametrize("name,func,old,new", RISE_MUTANTS, ids=[m[0] for m in RISE_MUTANTS])
def test_rise_edge_mutant_is_caught(name, func, old, new, monkeypatch):
    mod = _mutant_module(func, old, new, monkeypatch)
    monkeypatch.setattr(variant_pins, "O", mod)
    failed = []
    for pin in RISE_PINS:
        try:
            pin()
        except Exception:
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"


PROFILE_MUTANTS = [
    ("profile_volume_inner_edge_twice", "profile", "(hi ** 3 - lo ** 3)", "(lo ** 3 - lo ** 3 / 8.0)"),
    ("profile_volume_outer_only", "profile", "(hi ** 3 - lo ** 3)", "(hi ** 3)"),
    ("profile_closed_lower_edge", "profile", "(r_sorted > lo) & (r_sorted <= hi)", "(r_sorted >= lo) & (r_sorted <= hi)"),
    ("profile_vc_inner_edge", "profile", "math.sqrt(G * mass_in / hi)", "math.sqrt(G * mass_in / lo)"),
    ("profile_exclusive_mass", "profile", "m_sorted[r_sorted <= hi].sum()", "m_sorted[r_sorted < hi].sum()"),
]

PROFILE_PINS = [pins.test_profile_two_bins_hand_worked, pins.test_profile_counts_and_mass]


@pytest.mark.parametrize("name,func,old,new", PROFILE_MUTANTS, ids=[m[0] for m in PROFILE_MUTANTS])
def test_profile_mutant_is_caught(name, func, old, new, monkeypatch):
    mod = _mutant_module(func, old, new, monkeypatch)
    monkeypatch.setattr(pins, "O", mod)
    failed = []
    for pin in PROFILE_PINS:
        try:
            pin()
        except Exception:
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"
