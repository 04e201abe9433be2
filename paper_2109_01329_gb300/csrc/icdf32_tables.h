// Generated by gen_icdf32_tables.py (mpmath, 100-bit); do not edit.
// z = x P1(v) for v < V1, x P2(sqrt(v) - sqrt(V1)) above; fit errors with
// float coefficients 3.4e-08 and 7.0e-08 of max(1, |z|).
#pragma once
#define GRNG_ICDF32_V1 7.213475227355957f
#define GRNG_ICDF32_SQRT_V1 2.685791254043579f
#define GRNG_ICDF32_P1(v) \
  fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(-4.524745023104515e-10f, (v), 1.6423307158675016e-08f), (v), -2.114626340699033e-07f), (v), 5.973052452645788e-07f), (v), 1.0216094779025298e-05f), (v), -4.2003066482720897e-05f), (v), -0.0010987052228301764f), (v), 0.007846237160265446f), (v), 0.2274337261915207f), (v), 1.2533141374588013f)
#define GRNG_ICDF32_P2(d) \
  fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(-8.314958540722728e-05f, (d), 0.0006541353650391102f), (d), -0.0015712728491052985f), (d), -0.0014002003008499742f), (d), 0.016585253179073334f), (d), -0.044227033853530884f), (d), 0.06719748675823212f), (d), 1.1252485513687134f), (d), 2.9412994384765625f)
