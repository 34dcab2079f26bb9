"""Planted mistakes: each case copies the oracle's C source, plants one plausible slip (a cell
width of the wrong direction, a dropped wall velocity, a flipped sign, the wrong component or
split stage), builds the copy and runs the pins that must catch it.  A pin that still passes on
a planted mistake would leave the oracle, and with it every parity claim, unchecked there.

The slips are chosen where the other pins are blind: every earlier 2D pin holds under a dx
taken for dy (conservation telescopes whatever the width, symmetry pins are symmetric, a
global Maxwellian has no transport), and the mirror-symmetry pin of two facing diffuse walls
holds under any mistake made alike on both walls.
"""
import concurrent.futures as cf

import pytest

import test_oracle_pins as P
from oracle import build as B
from oracle import oracle as O

C = "mm_oracle.c"

# (name, [(old, new)], pins that must fail: (callable, kwargs))
MUTANTS = [
    ("micro y sweep with dx",
     [("double h = dir == 1 ? dx : dy;", "double h = dir == 1 ? dx : dx;")],
     [(P.test_free_streaming_along_y, {})]),
    ("macro y transport with dx",
     [("double v = Q2[m * nc + c] - dt / dy * (FT[m] - FB[m]);",
       "double v = Q2[m * nc + c] - dt / dx * (FT[m] - FB[m]);")],
     [(P.test_free_streaming_along_y, {}), (P.test_free_streaming_diagonal_unequal_cells, {})]),
    ("y heat-flux differences with dx",
     [("if (m >= 3) v -= dt * (dH[m - 3] / dy);", "if (m >= 3) v -= dt * (dH[m - 3] / dx);")],
     [(P.test_free_streaming_along_y, {}), (P.test_free_streaming_diagonal_unequal_cells, {})]),
    ("Ghat temperature gradient in y with dx",
     [("double dTdy = (Tface_yp - Tface_ym) / dy;", "double dTdy = (Tface_yp - Tface_ym) / dx;")],
     [(P.test_ghat_transport_term_converges_to_analytic_projection, {})]),
    ("Ghat strain s12 with dx for the y difference",
     [("double s12 = Dy_u1 / dy + Dx_u2 / dx;", "double s12 = Dy_u1 / dx + Dx_u2 / dx;")],
     [(P.test_ghat_transport_term_converges_to_analytic_projection, {})]),
    ("micro wall Maxwellian without U (x walls)",
     [("e = (v1 * v1 + (v2 - U) * (v2 - U)) / (2.0 * Tw);", "e = (v1 * v1 + v2 * v2) / (2.0 * Tw);")],
     [(P.test_diffuse_wall_micro_shear_closed_form, {"side": 0, "keep": 1}),
      (P.test_diffuse_wall_micro_shear_closed_form, {"side": 1, "keep": 0})]),
    ("micro wall Maxwellian without U (y walls)",
     [("e = ((v1 - U) * (v1 - U) + v2 * v2) / (2.0 * Tw);", "e = (v1 * v1 + v2 * v2) / (2.0 * Tw);")],
     [(P.test_diffuse_wall_micro_shear_closed_form, {"side": 2, "keep": 1}),
      (P.test_diffuse_wall_micro_shear_closed_form, {"side": 3, "keep": 0})]),
    ("micro wall density from P11 at y walls",
     [("rw = pc->rho * orc_wall_R(pc->u2, pc->P22 / pc->rho, Tw, s == 2 ? -1 : +1);",
       "rw = pc->rho * orc_wall_R(pc->u2, pc->P11 / pc->rho, Tw, s == 2 ? -1 : +1);")],
     [(P.test_diffuse_wall_micro_shear_closed_form, {"side": 2, "keep": 0})]),
    ("wall-cell ES term with the wrong sign",
     [("val += (gauss_es(pc, vel1(g, k), vel2(g, l)) - M[id]) / eps;",
       "val -= (gauss_es(pc, vel1(g, k), vel2(g, l)) - M[id]) / eps;")],
     [(P.test_diffuse_wall_micro_shear_closed_form, {"side": 1, "keep": 1})]),
    ("macro wall ghost without U (y walls)",
     [("gu1 = U; gu2 = 0.0;", "gu1 = 0.0; gu2 = 0.0;")],
     [(P.test_diffuse_wall_macro_step_closed_form, {"side": 2}),
      (P.test_diffuse_wall_macro_step_closed_form, {"side": 3})]),
    ("macro wall ghost without U (x walls)",
     [("gu1 = 0.0; gu2 = U;", "gu1 = 0.0; gu2 = 0.0;")],
     [(P.test_diffuse_wall_macro_step_closed_form, {"side": 0})]),
    ("macro wall density from P11 at y walls",
     [("rw = rho * orc_wall_R(u2, P22 / rho, Tw, side == 2 ? -1 : +1);",
       "rw = rho * orc_wall_R(u2, P11 / rho, Tw, side == 2 ? -1 : +1);")],
     [(P.test_diffuse_wall_macro_step_closed_form, {"side": 3})]),
    ("macro wall density with the side's sign flipped",
     [("rw = rho * orc_wall_R(u2, P22 / rho, Tw, side == 2 ? -1 : +1);",
       "rw = rho * orc_wall_R(u2, P22 / rho, Tw, side == 2 ? +1 : -1);")],
     [(P.test_diffuse_walls_conserve_mass, {})]),
    ("x transport from the state before the collision half step",
     [("face_flux_x(g, p, Q1, i, j, FL);", "face_flux_x(g, p, Q, i, j, FL);")],
     [(P.test_diffuse_wall_macro_step_closed_form, {"side": 0})]),
    ("full heat flux of the cell at a diffuse wall face",
     [("    default: return 0.5 * hc;\n  }\n}\nstatic double face_H_y",
       "    default: return hc;\n  }\n}\nstatic double face_H_y")],
     [(P.test_diffuse_wall_macro_step_closed_form, {"side": 1})]),
]


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    root = tmp_path_factory.mktemp("mutants")

    def one(k):
        return B.build_variant(str(root / ("m%02d" % k)), {C: MUTANTS[k][1]})

    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        return list(ex.map(one, range(len(MUTANTS))))


@pytest.mark.parametrize("k", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(builds, k):
    name, _, pins = MUTANTS[k]
    with O.use_library(builds[k]):
        for pin, kw in pins:
            with pytest.raises((AssertionError, O.OracleError)):
                pin(**kw)


def test_unplanted_copy_passes_the_same_pins(tmp_path):
    """The copy built without edits passes every pin used above, so a failure on a mutant is the
    planted mistake's doing."""
    path = B.build_variant(str(tmp_path / "clean"), {})
    seen = set()
    with O.use_library(path):
        for _, _, pins in MUTANTS:
            for pin, kw in pins:
                key = (pin.__name__, tuple(sorted(kw.items())))
                if key not in seen:
                    seen.add(key)
                    pin(**kw)
