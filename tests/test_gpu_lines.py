"""Several lines in one launch (irt_forward_ppv_lines) and the radial view of
an observer-centred [r][b][l] tensor (view.trilinear = 2), against the
single-line renders and the FP64 oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from synth import DUST, LINE_13CO_21, VelocityAxis, View, make_fields, to_storage  # noqa: E402
from synth.levels import rotor_model  # noqa: E402
from tests.gpu_helpers import COMP, assert_parity, torch_fields  # noqa: E402

PC = 3.0856775814913673e18


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401


def rotor_lines(model, rs):
    """LTE line constants of radiative transitions rs of a rigid-rotor model
    (13CO 1-0, 2-1, 3-2 for rs = 0, 1, 2 with the 13CO rotational constant)."""
    out = []
    b0 = float(model["nu_hz"][0]) / 2.0
    for r in rs:
        u, l = int(model["rad_up"][r]), int(model["rad_lo"][r])
        ln = dict(LINE_13CO_21)
        ln.update(nu_ul_hz=float(model["nu_hz"][r]), a_ul_s=float(model["a_ul_s"][r]),
                  e_u_k=float(model["energy_k"][u]), b0_hz=b0, g_u=float(model["g"][u]),
                  g_l=float(model["g"][l]))
        out.append(ln)
    return out


#: one dust opacity per line (Sec. 3.2 allows a kappa per line)
DUSTS = [dict(DUST, kappa_cm2_per_g_gas=k) for k in (0.004, 0.01, 0.02)]


def _all_pix(nx, ny):
    py, px = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([px.ravel(), py.ravel()], axis=1)


@pytest.mark.parametrize("integration", ["smooth", "formal", "formal_kahan"])
def test_three_lines_in_one_launch_equal_single_line_renders(integration):
    import paper_2607_01338_b300 as irt
    n = 24
    fs = make_fields(n, 41)
    st, deq = to_storage(fs, np.float32)
    dx = 0.1 * PC
    lines = rotor_lines(rotor_model(nlev=8), [0, 1, 2])
    va = VelocityAxis(80, -80.0, 2.0, 1)
    g = irt.Grid(*torch_fields(st), dx)
    for view in (View(0.0, 0.0, n, n, dx, 0), View(math.radians(30), math.radians(45), n, n, dx, 1)):
        multi = irt.forward_lines(g, view, va, lines, DUSTS, integration=integration)
        singles = [irt.forward(g, view, va, ln, du, integration=integration)
                   for ln, du in zip(lines, DUSTS)]
        torch.cuda.synchronize()
        for m, s in zip(multi, singles):
            peak = float(s["T"].abs().max())
            for k in COMP:
                d = float((m[k] - s[k]).abs().max())
                assert d <= 1e-6 * peak, (k, d, peak)
        # each line against the oracle
        pix = _all_pix(n, n)
        mode = oracle.SMOOTH if integration == "smooth" else oracle.FORMAL
        for m, ln, du in zip(multi, lines, DUSTS):
            orc = oracle.render(deq.as_tuple(), dx, ln, du, view, va, pix, integration=mode)
            gpu = {k: m[k].double().cpu().numpy() for k in COMP}
            assert_parity(gpu, orc, pix)
    g.close()


def test_lines_with_an_ot_grid_and_16bit_storage():
    """Three lines of one OT level-balance grid rendered together from fp16/bf16
    fields with an H2 abundance field, against the oracle per line."""
    import paper_2607_01338_b300 as irt
    n = 20
    m = rotor_model(nlev=20, seed=4)
    axes = dict(n_n=16, n_chi=6, n_t=12, log10_nh_min=1.0, log10_nh_max=7.5, chi_min=0.05,
                chi_max=0.5, log10_t_min=math.log10(8.0), log10_t_max=math.log10(300.0))
    tab = irt.LevelTable(m, axes, [0, 1, 2])
    otab = oracle.OTTable(m, axes, [0, 1, 2])
    fs = make_fields(n, 43)
    scales = [1e4, 1.0, 1.0, 1.0, 1e-6]
    st, deq = to_storage(fs, ["bf16", "bf16", "bf16", np.float16, np.float16], scales=scales)
    chi = np.random.default_rng(2).uniform(0.1, 0.5, (n, n, n)).astype(np.float16)
    dx = 0.1 * PC
    g = irt.Grid(*torch_fields(st), dx, scales=scales)
    g.set_h2_fraction(torch.from_numpy(chi).cuda())
    lines = rotor_lines(m, [0, 1, 2])
    va = VelocityAxis(64, -64.0, 2.0, 1)
    view = View(math.radians(50), math.radians(120), n, n, dx, 1)
    multi = irt.forward_lines(g, view, va, lines, DUSTS, levels=tab, line_indices=[0, 1, 2])
    torch.cuda.synchronize()
    pix = _all_pix(n, n)
    for q, (mc, ln, du) in enumerate(zip(multi, lines, DUSTS)):
        orc = oracle.render(deq.as_tuple(), dx, ln, du, view, va, pix, levels=otab,
                            line_index=q, chi=chi.astype(np.float64))
        assert float(np.abs(orc["L"]).max()) > 0.1
        gpu = {k: mc[k].double().cpu().numpy() for k in COMP}
        assert_parity(gpu, orc, pix)
    g.close()
    tab.close()
    otab.close()


def test_lines_argument_errors():
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300.binding import IRT_EINVAL, IRT_EUNSUPPORTED, IrtError
    n = 8
    st, _ = to_storage(make_fields(n, 3), np.float32)
    dx = 0.1 * PC
    g = irt.Grid(*torch_fields(st), dx)
    va = VelocityAxis(16, -16.0, 2.0, 1)
    view = View(0.0, 0.0, n, n, dx, 0)
    lines = rotor_lines(rotor_model(nlev=8), [0, 1, 2, 3, 4])
    with pytest.raises(IrtError) as e:
        irt.forward_lines(g, view, va, lines, [DUST] * 5)
    assert e.value.status == IRT_EUNSUPPORTED
    with pytest.raises(IrtError) as e:
        irt.forward_lines(g, View(0.0, 0.0, n + 1, n, dx, 0), va, lines[:2], [DUST] * 2)
    assert e.value.status == IRT_EINVAL
    g.close()


def test_radial_view_equals_z_view_of_the_reversed_tensor_and_the_oracle():
    """The [r][b][l] tensor read with view.trilinear = 2 renders exactly as the
    z view of the same tensor reversed along r; both against the oracle."""
    import paper_2607_01338_b300 as irt
    nr, nb, nl = 40, 12, 16
    fs = make_fields(40, 17)
    arrs = [np.ascontiguousarray(a[:nr, :nb, :nl]) for a in fs.as_tuple()]
    st = [a.astype(np.float32) for a in arrs]
    dr = 0.05 * PC
    va = VelocityAxis(96, -96.0, 2.0, 1)
    g = irt.Grid(*[torch.from_numpy(a).cuda() for a in st], dr)
    rev = irt.Grid(*[torch.from_numpy(np.ascontiguousarray(a[::-1])).cuda() for a in st], dr)
    rad = irt.forward(g, View(0.0, 0.0, nl, nb, dr, 2), va, LINE_13CO_21, DUST)
    zv = irt.forward(rev, View(0.0, 0.0, nl, nb, dr, 0), va, LINE_13CO_21, DUST)
    torch.cuda.synchronize()
    for k in COMP:
        assert torch.equal(rad[k], zv[k]), k
    pix = _all_pix(nl, nb)
    orc = oracle.render(tuple(a.astype(np.float64) for a in st), dr, LINE_13CO_21, DUST,
                        View(0.0, 0.0, nl, nb, dr, 2), va, pix)
    gpu = {k: rad[k].double().cpu().numpy() for k in COMP}
    assert_parity(gpu, orc, pix)
    # the thin modes read the same columns
    thin = irt.forward(g, View(0.0, 0.0, nl, nb, dr, 2), va, LINE_13CO_21, DUST,
                       transfer="selectively_thin")
    torch.cuda.synchronize()
    orc = oracle.render(tuple(a.astype(np.float64) for a in st), dr, LINE_13CO_21, DUST,
                        View(0.0, 0.0, nl, nb, dr, 2), va, pix,
                        transfer=oracle.SELECTIVELY_THIN)
    assert_parity({k: thin[k].double().cpu().numpy() for k in COMP}, orc, pix)
    g.close()
    rev.close()


def test_radial_view_adjoint_equals_the_reversed_z_view_adjoint():
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300.binding import IRT_FLAG_SAVE_CHECKPOINTS
    nr, nb, nl = 48, 8, 10
    fs = make_fields(48, 23)
    st = [np.ascontiguousarray(a[:nr, :nb, :nl]).astype(np.float32) for a in fs.as_tuple()]
    dr = 0.05 * PC
    va = VelocityAxis(64, -64.0, 2.0, 1)
    g = irt.Grid(*[torch.from_numpy(a).cuda() for a in st], dr)
    rev = irt.Grid(*[torch.from_numpy(np.ascontiguousarray(a[::-1])).cuda() for a in st], dr)
    vr, vz = View(0.0, 0.0, nl, nb, dr, 2), View(0.0, 0.0, nl, nb, dr, 0)
    L = irt.forward(g, vr, va, LINE_13CO_21, DUST, flags=IRT_FLAG_SAVE_CHECKPOINTS)["L"]
    cot = {"L": 1e-3 * L}
    gr = irt.adjoint(g, vr, va, LINE_13CO_21, DUST, cot)
    gz = irt.adjoint(rev, vz, va, LINE_13CO_21, DUST, cot)
    torch.cuda.synchronize()
    for a, b in zip(gr, gz):
        assert torch.allclose(a, torch.flip(b, dims=[0]), rtol=1e-5,
                              atol=1e-6 * float(b.abs().max()))
    g.close()
    rev.close()
