"""Plant plausible mistakes in copies of the oracle (on the CPU) and check that
the pins catch every one: each mutant must fail at least one pin."""
import os
import subprocess

import pytest

from oracle import oracle as O
from oracle import build_oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(build_oracle.__file__), "oracle.c")

MUTANTS = {
    "sqrt_term_sign": ("double F = kd - gs;", "double F = kd + gs;"),
    "rbar_formula": ("double rbar = (ri * rj) / (ri + rj);", "double rbar = (ri + rj) / 2.0;"),
    "cutoff_not_strict": ("if (!(d2 < R2)) continue;", "if (!(d2 <= R2)) continue;"),
    "accumulate_sign": ("a->fx = a->fx + sc * ddx;", "a->fx = a->fx - sc * ddx;"),
    "transposed_difference": ("double ddx = xi - st->x[j]", "double ddx = st->x[j] - xi"),
    "morton_axes_swapped": ("c |= ((y >> b) & 1ULL) << (3 * b + 1);", "c |= ((y >> b) & 1ULL) << (3 * b + 2);"),
    "no_grid_margin": ("g->lo[d] = floor(mn[d] / P->L) * P->L - P->L;", "g->lo[d] = floor(mn[d] / P->L) * P->L;"),
    "static_two_contacts": ("st->nz[i] > 1", "st->nz[i] > 2"),
    "static_ignores_old_position": ("dirty[ndirty++] = G.base[s] + box_linear(g, ox, oy, oz);", "(void)0;"),
    "cbrt_too_few_steps": ("it < 6", "it < 2"),
    "philox_weyl_constant": ("W0 = 0x9E3779B97F4A7C15ULL", "W0 = 0x9E3779B97F4A7C17ULL"),
    "daughter_uid_offset": ("st->next_uid + (uint64_t)rank;", "st->next_uid + (uint64_t)rank + 1;"),
    "mother_volume": ("double v1 = (v * rho) / (1.0 + rho);", "double v1 = v / (1.0 + rho);"),
    "clamp_missing": ("if (dn > P->dmax) {", "if (dn > 1e300) {"),
    "tolerance_base_signed": ("a->scale_abs += fabs(F);", "a->scale_abs += F;"),
    "tolerance_base_terms": ("a->scale_abs += fabs(F);", "a->scale_abs += kd + gs;"),
    "removal_no_swaps": ("for (int64_t e = 0; e < swaps; ++e) move_agent(st, to_left[e], to_right[e]);",
                         "(void)swaps;"),
    "removal_tail_descending": ("to_left[swaps_left++] = e + new_size;",
                                "to_left[swaps_left++] = new_size + removed - 1 - e;"),
    "removal_ghosts_ignored": ("dirty[ndirty++] = G.base[0] + box_linear(g, ox, oy, oz);", "(void)0;"),
    "death_ignores_behaviour": ("if ((st->beh[i] & BEH_DIE) && P->death_prob > 0.0)", "if (P->death_prob > 0.0)"),
    "removal_moves_keep_old_uid": ("  st->uid[to] = st->uid[from];\n", "\n"),
    "type_pair_own_type_twice": ("4u * TYPE_OF(st->beh[i]) + TYPE_OF(st->beh[j])",
                                 "4u * TYPE_OF(st->beh[i]) + TYPE_OF(st->beh[i])"),
    "type_gamma_from_k_table": ("gamma = P->type_gamma[ab];", "gamma = P->type_k[ab];"),
    "type_bits_shifted": ("#define TYPE_OF(beh) (((beh) >> 4) & 3u)", "#define TYPE_OF(beh) (((beh) >> 3) & 3u)"),
    "hilbert_no_reflection": ("X[0] ^= P; /* reflect the lower bits of axis 0 */", "(void)P;"),
    "hilbert_no_exchange": ("        X[i] ^= t;\n      }", "      }"),
    "hilbert_no_final_flip": ("  for (int i = 0; i < 3; ++i) X[i] ^= t;\n  uint64_t h = 0;", "  uint64_t h = 0;"),
    "hilbert_gray_order": ("  X[1] ^= X[0]; /* Gray encode */\n  X[2] ^= X[1];", "  X[2] ^= X[1]; /* Gray encode */\n  X[1] ^= X[0];"),
}


def _checks():
    c = []
    for row in pins._pair_lines():
        c.append(lambda row=row: pins.test_two_sphere_hand_worked(*row))
    for row in pins._scale_lines():
        c.append(lambda row=row: pins.test_tolerance_bases_two_spheres_hand_worked(*row))
    for row in pins._removal_lines():
        c.append(lambda row=row: pins.test_parallel_removal_hand_worked(*row))
    for seed in (1, 2):
        c.append(lambda seed=seed: pins.test_parallel_removal_invariants(seed))
    for row in pins._hetero_lines():
        c.append(lambda row=row: pins.test_heterotypic_two_spheres_hand_worked(*row))
    for bits in (2, 3):
        c.append(lambda bits=bits: pins.test_hilbert_is_a_face_adjacent_bijection(bits))
    for kind in ("uniform", "lattice_ties", "clustered"):
        c.append(lambda kind=kind: pins.test_grid_neighbors_equal_brute_force(kind))
    for key, ctr in [((5, 7), (0, 0, 0, 0)), ((2**64 - 1, 123), (2**64 - 1, 3, 9, 1))]:
        c.append(lambda key=key, ctr=ctr: pins.test_philox_matches_numpy_bit_generator(key, ctr))
    for dims in [(5, 2, 7), (3, 5)]:
        c.append(lambda dims=dims: pins.test_morton_offsets_against_brute_force(dims))
    for name in dir(pins):
        f = getattr(pins, name)
        if name.startswith("test_") and callable(f) and f.__code__.co_argcount == 0:
            c.append(f)
    return c


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not unique: %s" % name
    mpath = tmp_path / "oracle_mutant.c"
    mpath.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run([os.environ.get("CC", "cc")] + [f for f in build_oracle.CFLAGS if f != "-Wall"]
                   + [str(mpath), "-o", str(lib), "-lm"], check=True)
    failures = 0
    with O.use_library(str(lib)):
        for chk in _checks():
            try:
                chk()
            except Exception:
                failures += 1
    assert failures > 0, "mutant %s survived every pin" % name
