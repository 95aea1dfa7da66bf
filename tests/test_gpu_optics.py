"""Parity of the last-mile ray tracing (Sec. 6.4) with the FP64 oracle: the
kernel traces every photon that hits a telescope sphere through the parabolic
mirror onto its camera, photon by photon against the oracle's pixels, with
camera images equal to the records they summarise, on the planar and the
spherical path, through the host, device and streamed calls."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import binding as B
from paper_2405_04229_gb300 import synth
from tests import parity_util as PU

pytestmark = pytest.mark.gpu

ORC_ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
# 7 m mirror, 8 m focal length, 1 m camera of 41 x 41 pixels, pointing at the showers
OPT = dict(mirror_d=7.0, focal_f=8.0, camera_r=0.5, point_zenith=math.radians(20.0),
           point_azimuth=math.radians(30.0), cam_n=41)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _tel():
    return synth.grid_telescopes(nx=6, ny=6, pitch=60.0, radius=6.0)


def _camera_close(g, o, bunch, nonempty=True):
    """GPU and oracle images differ at most by the bunches whose pixel,
    telescope or optics survival decision lies in the oracle's edge band."""
    rec = o["records"]
    flagged = ((rec["status"] == oracle.ST_LANDED) & (rec["tel"] >= 0) &
               ((rec["flags"] & (oracle.FL_TEL_EDGE | oracle.FL_OPTICS)) != 0))
    diff = np.abs(g["camera"].astype(np.int64) - o["camera"].astype(np.int64)).sum()
    assert diff <= 2 * bunch * int(flagged.sum()), (diff, int(flagged.sum()))
    assert o["camera"].sum() > 0 or not nonempty


@pytest.mark.parametrize("refr,trans", [(True, True), (False, False)])
def test_planar_camera_parity(refr, trans):
    segs = synth.shower_segments(20000, 20.0, 30.0, 1e12, seed=4)
    tel = _tel()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=refr, transmission=trans)
    det = B.Detector(tel=tel, optics=OPT)
    g = B.propagate_host(segs, atm, det, seed=1, bunch=2, records=True)
    o = oracle.propagate(segs, ORC_ATM, tel=tel, bunch=2, refraction=refr, transmission=trans, seed=1, optics=OPT)
    st = PU.compare(g, o, bunch=2)
    assert st["pix_hits"] > 500, st
    _camera_close(g, o, 2)
    # photons on a camera are a part of those on its sphere
    assert (g["camera"].sum(axis=(2, 3)) <= g["tel_counts"]).all()


def test_spherical_camera_parity():
    """Inclined showers on the spherical shell; the sphere's ground points carry
    FP32 ulps of ~4 mm, so rim and pixel decisions are flagged within 3 cm and
    the camera is coarser (5 x 5 pixels of 20 cm)."""
    opt = dict(OPT, cam_n=5, point_zenith=math.radians(20.0))
    segs = synth.shower_segments(15000, 20.0, 30.0, 1e13, seed=6)
    tel = _tel()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True, spherical=True)
    det = B.Detector(tel=tel, spherical=True, optics=opt)
    g = B.propagate_host(segs, atm, det, seed=2, bunch=2, records=True)
    o = oracle.propagate(segs, ORC_ATM, tel=tel, bunch=2, refraction=True, transmission=True, seed=2,
                         spherical=True, optics=opt, bands=dict(band_pos=0.03))
    st = PU.compare(g, o, bunch=2)
    assert st["pix_hits"] > 250, st
    _camera_close(g, o, 2)


def test_camera_off_axis_pointing_images_fewer_photons():
    """A telescope pointing 10 degrees away from the showers (beyond the
    camera's 3.6-degree half field of view) images few of their photons: the
    kernel follows the pointing, as the oracle does."""
    segs = synth.shower_segments(10000, 20.0, 30.0, 1e12, seed=8)
    tel = _tel()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=False)
    on = B.propagate_host(segs, atm, B.Detector(tel=tel, optics=OPT), seed=3, bunch=2)
    off_opt = dict(OPT, point_zenith=math.radians(30.0))
    off = B.propagate_host(segs, atm, B.Detector(tel=tel, optics=off_opt), seed=3, bunch=2)
    o = oracle.propagate(segs, ORC_ATM, tel=tel, bunch=2, refraction=True, seed=3, optics=off_opt)
    assert np.array_equal(on["tel_counts"], off["tel_counts"])   # spheres do not depend on the pointing
    assert off["camera"].sum() < 0.5 * on["camera"].sum()
    _camera_close(off, o, 2, nonempty=False)


def test_device_and_streamed_calls_fill_the_camera():
    """Device outputs and the streamed path (chunks accumulating on two
    streams) give the host call's camera images exactly."""
    torch = pytest.importorskip("torch")
    segs = synth.shower_segments(9000, 20.0, 30.0, 1e12, seed=9)
    arr = B.pack_segments(segs)
    tel = _tel()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(tel=tel, optics=OPT)
    ref = B.propagate_host(segs, atm, det, seed=5, bunch=3)
    assert ref["camera"].sum() > 0
    pinned = torch.from_numpy(arr.view(np.uint8)).pin_memory()
    outs = B.DeviceOutputs(det)
    st = B.Streamer(2_000)
    for _ in range(2):   # the second run re-zeroes the camera
        st.run(pinned.data_ptr(), len(arr), atm, det, outs.out, seed=5, bunch=3)
        h = outs.host()
        assert np.array_equal(h["camera"], ref["camera"])
        assert np.array_equal(h["tel_counts"], ref["tel_counts"])
    st.close()


def test_missing_camera_output_and_small_spheres_are_rejected():
    torch = pytest.importorskip("torch")
    tel = _tel()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=False, transmission=False)
    det = B.Detector(tel=tel, optics=OPT)
    outs = B.DeviceOutputs(det)
    outs.out.camera = None
    segs = torch.from_numpy(B.pack_segments(synth.shower_segments(10, 20.0, 0.0, 1e12, seed=0)).view(np.uint8)).cuda()
    o = B.cs_opts_default()
    o.device_ptrs, o.bunch = 1, 1
    assert B.cs_propagate_ex(segs.data_ptr(), 10, atm.handle, det.handle, 0, o, outs.out) == B.CS_ERR_INVALID_ARG
    small = np.array(tel)
    small[:, 3] = 5.0   # below sqrt(3.5^2 + 4^2) = 5.32 m: the sphere would cut the instrument
    with pytest.raises(RuntimeError):
        B.Detector(tel=small, optics=OPT)
    with pytest.raises(RuntimeError):
        B.Detector(tel=tel, optics=dict(OPT, focal_f=0.0))


# mirror reflectivity and camera efficiency (a synthetic stand-in for a coated
# mirror and a photomultiplier camera)
EFF = dict(lambda_nm=[300.0, 350.0, 420.0, 500.0, 600.0],
           mirror=[0.80, 0.86, 0.90, 0.89, 0.87],
           camera=[0.18, 0.26, 0.24, 0.15, 0.05])


@pytest.mark.parametrize("spherical", [False, True])
def test_camera_absorption_parity(spherical):
    """Absorption in the optics (Sec. 6.4): the camera keeps each photon with
    probability R(lambda) eps(lambda) by its own keyed draw; pixels photon by
    photon against the oracle, images equal to the records, and every kept
    photon a photon of the lossless run's image."""
    # on the sphere the camera is coarser (5 x 5 pixels): ground points carry FP32 ulps of ~4 mm
    opt = dict(OPT, efficiency=EFF, cam_n=5 if spherical else 41)
    free_opt = dict(OPT, cam_n=opt["cam_n"])
    if spherical:
        segs = synth.shower_segments(20000, 20.0, 30.0, 1e13, seed=8)
        atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True, spherical=True)
    else:
        segs = synth.shower_segments(20000, 20.0, 30.0, 1e12, seed=7)
        atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    tel = _tel()
    det = B.Detector(tel=tel, optics=opt, spherical=spherical)
    free_det = B.Detector(tel=tel, optics=free_opt, spherical=spherical)
    g = B.propagate_host(segs, atm, det, seed=3, bunch=1, records=True)
    free = B.propagate_host(segs, atm, free_det, seed=3, bunch=1, records=True)
    bands = dict(band_pos=0.03) if spherical else None
    o = oracle.propagate(segs, ORC_ATM, tel=tel, bunch=1, refraction=True, transmission=True, seed=3, optics=opt,
                         spherical=spherical, bands=bands)
    st = PU.compare(g, o, bunch=1)
    assert st["pix_hits"] > 100, st
    _camera_close(g, o, 1)
    assert (g["camera"] <= free["camera"]).all()
    kept, seen = g["camera"].sum(), free["camera"].sum()
    assert 0.05 * seen < kept < 0.4 * seen, (kept, seen)
