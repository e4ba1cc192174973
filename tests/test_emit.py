"""The generated coefficient headers (csrc/boys_coeffs_f64.inc and
boys_coeffs_f32.inc: root products, constants and the exponential's tables)
are exactly what fit/emit.py writes from the committed fits, so a change to
either side shows here."""
import os

from paper_2504_07637_gb300.fit import emit


def _read(name):
    with open(os.path.join(emit.CSRC, name)) as fh:
        return fh.read()


def test_f64_header_is_the_generators_output():
    assert emit.render_f64() == _read("boys_coeffs_f64.inc")


def test_f32_header_is_the_generators_output():
    src = emit.render_f32()
    assert src is not None and src == _read("boys_coeffs_f32.inc")
