"""Seeded synthetic ionospheres and ray fans shaped like the paper's workloads.

This module is *input*, not method: it samples analytic electron-density
profiles onto uniform lat/lon/alt grids and describes ray fans.  Both the CUDA
path and the CPU oracle consume what it produces; it holds none of the
tracer's arithmetic (no interpolation, no refractive index, no integration).

The paper drives its experiments with IRI-2020 densities and IGRF-13 fields
(Sec. II-C, Sec. IV), which are not available here.  The stand-ins follow the
shapes it describes: an E layer near 110 km and an F2 layer near 300 km at
mid latitudes (Sec. IV-B), frequencies of 8-15 MHz and elevation scans
(Table II), and a centred tilted dipole for the field.

Profiles are alpha-Chapman layers, Ne = Nm exp(1/2 (1 - z - e^-z)),
z = (h - hm)/H, with Nm = fo^2 / 80.6 (fo in Hz, Ne in m^-3).  A travelling
ionospheric disturbance (TID) multiplies Ne by
1 + A exp(-rho^2 / (2 sigma^2)) cos(2 pi s / lambda + phase), where rho is the
great-circle distance from the TID centre and s the distance along its
propagation azimuth; centre, azimuth and phase come from a seeded generator.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

EARTH_RADIUS_KM = 6371.0

MODE_O = 1
MODE_X = 2

RK4 = 0
RKF45 = 1

FP64 = 0
MIXED = 1


@dataclass
class GridSpec:
    """Uniform lat/lon/alt grid; samples are stored [lat][lon][alt], alt fastest."""

    n_lat: int
    n_lon: int
    n_alt: int
    lat0_deg: float
    lon0_deg: float
    alt0_km: float
    dlat_deg: float
    dlon_deg: float
    dalt_km: float
    earth_radius_km: float = EARTH_RADIUS_KM
    b0_tesla: float = 0.0
    pole_lat_deg: float = 90.0
    pole_lon_deg: float = 0.0

    @property
    def shape(self):
        return (self.n_lat, self.n_lon, self.n_alt)

    def axes(self):
        lat = self.lat0_deg + self.dlat_deg * np.arange(self.n_lat)
        lon = self.lon0_deg + self.dlon_deg * np.arange(self.n_lon)
        alt = self.alt0_km + self.dalt_km * np.arange(self.n_alt)
        return lat, lon, alt


@dataclass
class FanSpec:
    """A fan of rays: every (frequency, mode, elevation, azimuth) combination.

    Results come back in the canonical order [freq][mode][el][az], with the
    ordinary mode first when both modes are requested.
    """

    tx_lat_deg: float
    tx_lon_deg: float
    tx_alt_km: float
    freq_mhz: np.ndarray
    el_deg: np.ndarray
    az_deg: np.ndarray
    modes: int = MODE_O
    integrator: int = RK4
    h_km: float = 1.0
    rtol: float = 1e-8
    atol_km: float = 1e-6
    h_min_km: float = 1e-6
    h_max_km: float = 20.0
    max_steps: int = 100000
    max_group_path_km: float = 0.0
    precision: int = FP64

    def __post_init__(self):
        self.freq_mhz = np.ascontiguousarray(np.atleast_1d(self.freq_mhz), dtype=np.float64)
        self.el_deg = np.ascontiguousarray(np.atleast_1d(self.el_deg), dtype=np.float64)
        self.az_deg = np.ascontiguousarray(np.atleast_1d(self.az_deg), dtype=np.float64)

    @property
    def mode_list(self):
        """Mode signs in canonical order: +1 ordinary, -1 extraordinary."""
        out = []
        if self.modes & MODE_O:
            out.append(1)
        if self.modes & MODE_X:
            out.append(-1)
        return out

    @property
    def n_rays(self):
        return len(self.freq_mhz) * len(self.mode_list) * len(self.el_deg) * len(self.az_deg)

    def replace(self, **kw):
        return dataclasses.replace(self, **kw)

    def ray_params(self, idx):
        """(freq_mhz, mode_sign, el_deg, az_deg) of canonical ray index idx."""
        n_az, n_el, modes = len(self.az_deg), len(self.el_deg), self.mode_list
        a = idx % n_az
        e = (idx // n_az) % n_el
        m = (idx // (n_az * n_el)) % len(modes)
        f = idx // (n_az * n_el * len(modes))
        return self.freq_mhz[f], modes[m], self.el_deg[e], self.az_deg[a]


@dataclass
class Workload:
    name: str
    grid: GridSpec
    ne: np.ndarray  # float32 or float64, shape grid.shape
    fan: FanSpec
    notes: dict = field(default_factory=dict)


def nm_from_fo(fo_mhz):
    """Peak density (m^-3) of a layer with critical frequency fo (MHz)."""
    return (np.asarray(fo_mhz) * 1e6) ** 2 / 80.6


def chapman(alt_km, nm, hm_km, h_km):
    z = (alt_km - hm_km) / h_km
    return nm * np.exp(0.5 * (1.0 - z - np.exp(-z)))


def _great_circle_km(lat1, lon1, lat2, lon2, re=EARTH_RADIUS_KM):
    p1, p2 = np.radians(lat1), np.radians(lat2)
    dl = np.radians(lon2 - lon1)
    c = np.sin(p1) * np.sin(p2) + np.cos(p1) * np.cos(p2) * np.cos(dl)
    return re * np.arccos(np.clip(c, -1.0, 1.0))


def tid_factor(lat, lon, rng, amp=0.05, wavelength_km=200.0, sigma_km=600.0,
               centre=(30.0, 112.0), spread_deg=5.0, phase_shift=0.0):
    """Multiplicative TID perturbation on a (lat, lon) mesh (degrees).
    phase_shift (cycles) advances the wave: the same disturbance a little later."""
    lat_c = centre[0] + rng.uniform(-spread_deg, spread_deg)
    lon_c = centre[1] + rng.uniform(-spread_deg, spread_deg)
    direction = rng.uniform(0.0, 2.0 * np.pi)
    phase = rng.uniform(0.0, 2.0 * np.pi) + 2.0 * np.pi * phase_shift
    rho = _great_circle_km(lat_c, lon_c, lat, lon)
    dn = np.radians(lat - lat_c) * EARTH_RADIUS_KM
    de = np.radians(lon - lon_c) * EARTH_RADIUS_KM * np.cos(np.radians(lat_c))
    s = dn * np.cos(direction) + de * np.sin(direction)
    env = np.exp(-(rho ** 2) / (2.0 * sigma_km ** 2))
    return 1.0 + amp * env * np.cos(2.0 * np.pi * s / wavelength_km + phase), dict(
        lat_c=lat_c, lon_c=lon_c, direction=direction, phase=phase)


def centred_grid(tx_lat, tx_lon, n_lat, n_lon, n_alt, dlat, dlon, dalt, alt0=60.0, **kw):
    return GridSpec(n_lat=n_lat, n_lon=n_lon, n_alt=n_alt,
                    lat0_deg=tx_lat - dlat * (n_lat - 1) / 2.0,
                    lon0_deg=tx_lon - dlon * (n_lon - 1) / 2.0,
                    alt0_km=alt0, dlat_deg=dlat, dlon_deg=dlon, dalt_km=dalt, **kw)


def dipole_field(tx_lon, b0=3.1e-5, tilt_deg=11.0):
    """Dipole with 11 deg tilt; the pole sits on the meridian opposite the transmitter."""
    pole_lon = ((tx_lon + 180.0 + 180.0) % 360.0) - 180.0
    return dict(b0_tesla=b0, pole_lat_deg=90.0 - tilt_deg, pole_lon_deg=pole_lon)


def two_layer_ne(grid: GridSpec, rng, foe=3.0, hme=110.0, he=10.0, fof2_lo=6.0, fof2_hi=10.0,
                 hmf2=300.0, hf2=50.0, tid_amp=0.05, daynight=0.0, centre=(30.0, 112.0), tid_phase_shift=0.0):
    lat, lon, alt = grid.axes()
    LAT, LON, ALT = np.meshgrid(lat, lon, alt, indexing="ij")
    fof2 = fof2_lo + (fof2_hi - fof2_lo) * (LAT - lat[0]) / (lat[-1] - lat[0])
    ne = chapman(ALT, nm_from_fo(foe), hme, he) + chapman(ALT, nm_from_fo(fof2), hmf2, hf2)
    tid, info = tid_factor(LAT[:, :, 0], LON[:, :, 0], rng, amp=tid_amp, centre=centre, phase_shift=tid_phase_shift)
    ne = ne * tid[:, :, None]
    if daynight:
        half = 0.5 * (lon[-1] - lon[0])
        ne = ne * (1.0 + daynight * (LON - centre[1]) / half)
    return ne, info


TX = (30.0, 112.0, 0.0)  # transmitter of Table II case D1 (30 N, 112 E)


def config1(dtype=np.float64) -> Workload:
    """Isotropic FP64 case: one Chapman F2 layer (foF2 8 MHz, hmF2 300 km,
    H 60 km) on a 21x21x61 grid (2 deg, 2 deg, 10 km; 60-660 km) centred on
    the transmitter; one 10 MHz fan of 16 elevations 5-50 deg; RK4, h = 1 km."""
    g = centred_grid(TX[0], TX[1], 21, 21, 61, 2.0, 2.0, 10.0)
    _, _, alt = g.axes()
    prof = chapman(alt, nm_from_fo(8.0), 300.0, 60.0)
    ne = np.broadcast_to(prof, g.shape).astype(dtype).copy()
    fan = FanSpec(*TX, freq_mhz=[10.0], el_deg=np.linspace(5.0, 50.0, 16), az_deg=[30.0],
                  modes=MODE_O, integrator=RK4, h_km=1.0, max_steps=20000)
    return Workload("chapman-F2 isotropic 21x21x61, 16 rays, RK4 h=1 km", g, ne, fan)


def config2(seed=2, dtype=np.float32, elev_step=0.5, az_step=10.0, freqs=(8.0, 12.0, 16.0),
            tid_phase_shift=0.0) -> Workload:
    """Anisotropic O+X case: dipole (3.1e-5 T, 11 deg tilt); E layer (foE 3 MHz,
    110 km) + F2 with foF2 linear 6-10 MHz across latitude + 5 % / 200 km TID;
    91x181x151 grid (1 deg, 1 deg, 4 km) of FP32 samples; 8/12/16 MHz x
    elevations 3-60 deg step 0.5 x azimuths 0-350 step 10 x O and X
    (24,840 rays); RKF45, rtol 1e-8.  tid_phase_shift (cycles): a later
    snapshot, the TID advanced along its direction of travel."""
    rng = np.random.default_rng(seed)
    g = centred_grid(TX[0], TX[1], 91, 181, 151, 1.0, 1.0, 4.0, **dipole_field(TX[1]))
    ne, info = two_layer_ne(g, rng, tid_phase_shift=tid_phase_shift)
    fan = FanSpec(*TX, freq_mhz=np.array(freqs),
                  el_deg=np.arange(3.0, 60.0 + 1e-9, elev_step),
                  az_deg=np.arange(0.0, 360.0 - 1e-9, az_step),
                  modes=MODE_O | MODE_X, integrator=RKF45, h_km=1.0, rtol=1e-8, atol_km=1e-6,
                  h_min_km=1e-6, h_max_km=20.0, max_steps=200000)
    return Workload("E+F2+TID dipole 91x181x151 fp32, 3f x 115el x 36az x O/X, RKF45 rtol 1e-8",
                    g, ne.astype(dtype), fan, notes=dict(tid=info, seed=seed))


def config4(seed=4, dtype=np.float32, rtol=1e-8, tid_phase_shift=0.0) -> Workload:
    """Ionogram-synthesis batch: 181x361x301 grid (0.5 deg, 0.5 deg, 2 km),
    two-layer Chapman + TID + 20 % day/night gradient; 2-30 MHz step 0.1 x
    elevations 1-89 deg step 0.1 x O and X (495,122 rays); RKF45 at rtol
    1e-8, the anisotropic fan case's tolerance (the batch's accuracy is held
    to the same bar).  tid_phase_shift (cycles) gives a later snapshot of the
    same ionosphere: the TID advanced along its direction of travel."""
    rng = np.random.default_rng(seed)
    g = centred_grid(TX[0], TX[1], 181, 361, 301, 0.5, 0.5, 2.0, **dipole_field(TX[1]))
    ne, info = two_layer_ne(g, rng, daynight=0.2, tid_phase_shift=tid_phase_shift)
    fan = FanSpec(*TX, freq_mhz=np.round(np.arange(2.0, 30.0 + 1e-9, 0.1), 10),
                  el_deg=np.round(np.arange(1.0, 89.0 + 1e-9, 0.1), 10), az_deg=[45.0],
                  modes=MODE_O | MODE_X, integrator=RKF45, h_km=1.0, rtol=rtol, atol_km=1e-6,
                  h_min_km=1e-6, h_max_km=20.0, max_steps=200000)
    return Workload("two-layer+TID+day/night 181x361x301 fp32, 281f x 881el x O/X", g,
                    ne.astype(dtype), fan, notes=dict(tid=info, seed=seed))


def serving_grids(seeds=(5, 6, 7, 8)):
    """Four resident grids of differing sizes for the request loop."""
    shapes = [((21, 21, 61), (2.0, 2.0, 10.0)), ((61, 121, 101), (1.5, 1.5, 6.0)),
              ((91, 181, 151), (1.0, 1.0, 4.0)), ((181, 361, 301), (0.5, 0.5, 2.0))]
    out = []
    for seed, ((nl, nn, na), (dl, dn, da)) in zip(seeds, shapes):
        rng = np.random.default_rng(seed)
        g = centred_grid(TX[0], TX[1], nl, nn, na, dl, dn, da, **dipole_field(TX[1]))
        ne, _ = two_layer_ne(g, rng)
        out.append((g, ne.astype(np.float32)))
    return out


def sample_indices(n_total, n_sample, seed):
    """Seeded sample of ray indices (sorted, without replacement)."""
    rng = np.random.default_rng(seed)
    n_sample = min(n_sample, n_total)
    return np.sort(rng.choice(n_total, size=n_sample, replace=False))


SERVING_MAX_RAYS = 100_000


def serving_mean_rays(max_rays=SERVING_MAX_RAYS):
    """Expected size of a log-uniform request size on [1, max_rays]."""
    return (max_rays - 1.0) / np.log(max_rays)


def serving_requests(n, seed, grid_specs, max_rays=SERVING_MAX_RAYS):
    """Seeded stream of fan requests for the serving loop.

    Each request picks one of the resident grids, a transmitter within 5 deg
    of that grid's centre, one magnetoionic mode, and a target size drawn
    log-uniformly from 1..max_rays rays.  Half are ionogram-synthesis shaped
    (one azimuth, a list of 3-30 MHz frequencies x an elevation scan), half
    OTHR coordinate-registration shaped (one or two frequencies x an elevation
    x azimuth fan).  Integration as in the anisotropic fan case (RKF45,
    rtol 1e-8), mixed precision.  Returns a list of (grid index, FanSpec).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        gi = int(rng.integers(len(grid_specs)))
        g = grid_specs[gi]
        lat_c = g.lat0_deg + 0.5 * g.dlat_deg * (g.n_lat - 1)
        lon_c = g.lon0_deg + 0.5 * g.dlon_deg * (g.n_lon - 1)
        target = int(np.clip(np.round(np.exp(rng.uniform(0.0, np.log(max_rays)))), 1, max_rays))
        if rng.random() < 0.5:  # ionogram synthesis: frequencies x elevations, one azimuth
            n_freq = int(min(target, rng.integers(1, 65)))
            n_az = 1
        else:  # OTHR registration: one or two frequencies x elevation x azimuth
            n_freq = int(min(target, rng.integers(1, 3)))
            n_az = int(max(1, min(36, target // (8 * n_freq))))
            n_az = int(rng.integers(1, n_az + 1))
        n_el = max(1, int(np.ceil(target / (n_freq * n_az))))
        el_lo = rng.uniform(1.0, 30.0)
        el_hi = min(89.0, el_lo + rng.uniform(5.0, 60.0))
        az0 = rng.uniform(0.0, 360.0)
        az_span = rng.uniform(10.0, 120.0) if n_az > 1 else 0.0
        fan = FanSpec(tx_lat_deg=lat_c + rng.uniform(-5.0, 5.0), tx_lon_deg=lon_c + rng.uniform(-5.0, 5.0),
                      tx_alt_km=0.0, freq_mhz=np.sort(rng.uniform(3.0, 30.0, n_freq)),
                      el_deg=np.linspace(el_lo, el_hi, n_el),
                      az_deg=np.mod(az0 + np.linspace(0.0, az_span, n_az), 360.0),
                      modes=MODE_O if rng.random() < 0.5 else MODE_X, integrator=RKF45, h_km=1.0, rtol=1e-8,
                      atol_km=1e-6, h_min_km=1e-6, h_max_km=20.0, max_steps=200000, precision=MIXED)
        out.append((gi, fan))
    return out


def interp_comparison(seed=10, refine=4):
    """Inputs for the GD-versus-Catmull-Rom comparison (Sec. IV): one analytic
    ionosphere (E layer + F2 with a 6-10 MHz latitude gradient, a 5 % TID of
    600 km wavelength, the anisotropic fan case's dipole) sampled on a coarse
    grid (1 deg, 1 deg, 5 km; 31x31x121 over +-15 deg, 60-660 km) and on a
    grid `refine` times finer along every axis over the same box, which stands
    in for the analytic field.  Fan: 8 and 12 MHz x O/X x elevations 5-55 deg
    step 0.5 x azimuths 0-315 step 45 (3,232 rays), RKF45 rtol 1e-9.
    Returns (coarse GridSpec, coarse Ne, fine GridSpec, fine Ne, FanSpec)."""
    rng = np.random.default_rng(seed)
    tid_params = dict(lat_c=TX[0] + rng.uniform(-5.0, 5.0), lon_c=TX[1] + rng.uniform(-5.0, 5.0),
                      direction=rng.uniform(0.0, 2.0 * np.pi), phase=rng.uniform(0.0, 2.0 * np.pi))
    field = dipole_field(TX[1])
    lat_lo, lat_hi = TX[0] - 15.0, TX[0] + 15.0

    def sample(g):
        lat, lon, alt = g.axes()
        LAT, LON, ALT = np.meshgrid(lat, lon, alt, indexing="ij")
        fof2 = 6.0 + 4.0 * (LAT - lat_lo) / (lat_hi - lat_lo)
        ne = chapman(ALT, nm_from_fo(3.0), 110.0, 10.0) + chapman(ALT, nm_from_fo(fof2), 300.0, 50.0)
        la, lo = LAT[:, :, 0], LON[:, :, 0]
        rho = _great_circle_km(tid_params["lat_c"], tid_params["lon_c"], la, lo)
        dn = np.radians(la - tid_params["lat_c"]) * EARTH_RADIUS_KM
        de = np.radians(lo - tid_params["lon_c"]) * EARTH_RADIUS_KM * np.cos(np.radians(tid_params["lat_c"]))
        s = dn * np.cos(tid_params["direction"]) + de * np.sin(tid_params["direction"])
        tid = 1.0 + 0.05 * np.exp(-(rho ** 2) / (2.0 * 600.0 ** 2)) * np.cos(2.0 * np.pi * s / 600.0 +
                                                                           tid_params["phase"])
        return ne * tid[:, :, None]

    coarse = centred_grid(TX[0], TX[1], 31, 31, 121, 1.0, 1.0, 5.0, **field)
    fine = centred_grid(TX[0], TX[1], 30 * refine + 1, 30 * refine + 1, 120 * refine + 1,
                        1.0 / refine, 1.0 / refine, 5.0 / refine, **field)
    fan = FanSpec(*TX, freq_mhz=np.array([8.0, 12.0]), el_deg=np.arange(5.0, 55.0 + 1e-9, 0.5),
                  az_deg=np.arange(0.0, 360.0 - 1e-9, 45.0), modes=MODE_O | MODE_X, integrator=RKF45,
                  h_km=1.0, rtol=1e-9, atol_km=1e-6, h_min_km=1e-6, h_max_km=20.0, max_steps=200000)
    return coarse, sample(coarse), fine, sample(fine), fan
