"""Composite-polynomial coefficient tables, transcribed from the paper (oracle copy).

TEST INFRASTRUCTURE ONLY: part of the CPU FP64 oracle. Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import anything under ``oracle/``.

Every polynomial is odd and of degree 5 (Sec. 3.3 sets d_t = 5 for all t):
    f_t(x) = a_t x + b_t x^3 + c_t x^5,
stored here as (a_t, b_t, c_t).

* ``SINGLE_FSTAR`` / ``SINGLE_FTILDE`` -- Table 1 (single precision, eps = 1e-3,
  T = 10): the Stage-I sequential-Remez polynomials f*_t (Sec. 3.1,
  Algorithm 1) and the Stage-II gradient-refined polynomials f~*_t (Sec. 3.2).
* ``HALF_FSTAR`` / ``HALF_FTILDE`` -- Table 2 (half precision, eps = 1e-3, T = 7).

The run-time filter (Algorithm 2) uses the refined columns f~*.  The
finite-precision rescaling of Sec. 3.4 ("numerical instability") is given by
``post_scale``: the iterate produced by stage t is divided by s_t.
Reading used here (the paper says "at the end of every half-precision
iteration" for half and "after each of the first eight iterations" for
single): half divides after stages 1..T-1 (s_T = 1), single after stages
1..8.  Dividing the final half iterate as well would bias every positive
eigenvalue of the output by 0.5 %, which is inconsistent with the accuracy the
paper reports in Sec. 4.1; the scalar tests in ``tests/`` measure both
readings.

The printed e_float values (Tables 1 and 2) are kept in
``tests/golden/e_float.txt`` with their citations.
"""

# Table 1, column f*_single (Stage I, sequential Remez, Algorithm 1).
SINGLE_FSTAR = (
    (8.5098853026, -25.2643041908, 18.7535678997),
    (4.2495734789, -3.1549764881, 0.5858847825),
    (4.2251221908, -3.1380444351, 0.5839534551),
    (4.1248386870, -3.0683324528, 0.5760029536),
    (3.7580103358, -2.8092738924, 0.5464842066),
    (2.8561775413, -2.1340562332, 0.4701107692),
    (2.0206004158, -1.4037211505, 0.3906738969),
    (1.8758751005, -1.2509719905, 0.3750972123),
    (1.8750000000, -1.2500000000, 0.3750000000),
    (1.8750000000, -1.2500000000, 0.3750000000),
)

# Table 1, column f~*_single (Stage II, gradient refinement for ReLU).
SINGLE_FTILDE = (
    (8.3119043343, -23.0739115930, 16.4664144722),
    (4.1439360087, -2.9176674704, 0.5246212487),
    (4.0257813209, -2.9025002398, 0.5334261214),
    (3.5118574347, -2.5740236523, 0.5050097282),
    (2.4398158400, -1.7586675341, 0.4191290613),
    (1.9779835097, -1.3337358510, 0.3772169049),
    (1.9559726949, -1.3091355170, 0.3746734515),
    (1.9282822454, -1.2823649693, 0.3704626545),
    (1.9220135179, -1.2812524618, 0.3707011753),
    (1.8942192942, -1.2613293407, 0.3676616051),
)

# Table 2, column f*_half (Stage I).
HALF_FSTAR = (
    (8.4703288038, -25.1080747067, 18.6292755991),
    (4.1828341833, -3.1087011099, 0.5806066814),
    (3.9618572790, -2.9540637464, 0.5629761180),
    (3.2865862170, -2.4647201345, 0.5073576939),
    (2.2737499945, -1.6446603679, 0.4161909275),
    (1.8887161973, -1.2651572253, 0.3765189256),
    (1.8750008858, -1.2500009843, 0.3750000984),
)

# Table 2, column f~*_half (Stage II).
HALF_FTILDE = (
    (8.2885332412, -22.5927099246, 15.8201383114),
    (4.1666196466, -2.9679004036, 0.5307623217),
    (4.0611848147, -2.9698947955, 0.5492133813),
    (3.6678301399, -2.7561018955, 0.5421513305),
    (2.7632556383, -2.0607754898, 0.4695405857),
    (2.0527445797, -1.4345145882, 0.4070669182),
    (1.8804816691, -1.2583997294, 0.3779501813),
)

EPSILON = 1e-3  # Sec. 3.3: eps = 10^-3 for both settings.
LANCZOS_STEPS = 20  # Sec. 3.4 / Algorithm 2: 20-step Lanczos on X^2.


def post_scale(kind, T):
    """Per-stage divisors s_1..s_T of Sec. 3.4 (reading stated in the module doc).

    kind: "half" -> 1.01 after stages 1..T-1; "single" -> 1.001 after stages 1..8;
    "none" -> no rescaling.
    """
    if kind == "half":
        return tuple(1.01 if t < T else 1.0 for t in range(1, T + 1))
    if kind == "half_all":  # the literal alternative reading, kept for the tests
        return tuple(1.01 for _ in range(T))
    if kind == "single":
        return tuple(1.001 if t <= 8 else 1.0 for t in range(1, T + 1))
    if kind == "none":
        return tuple(1.0 for _ in range(T))
    raise ValueError(kind)


def schedule(name):
    """Named run-time schedules: list of (a, b, c) and the per-stage divisors.

    "half":   f~*_half (Table 2), T = 7, 22 GEMMs (3T + 1).
    "single": f~*_single (Table 1), T = 10, 31 GEMMs.
    """
    if name == "half":
        return HALF_FTILDE, post_scale("half", len(HALF_FTILDE))
    if name == "single":
        return SINGLE_FTILDE, post_scale("single", len(SINGLE_FTILDE))
    raise ValueError(name)
