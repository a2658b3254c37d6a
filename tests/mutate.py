"""Planting a mistake in the oracle, on the CPU, to show that a pin catches it.

`mutated(module, name, old, new)` returns a copy of the function `name` of the
oracle module with the source text `old` replaced by `new` (exactly one
occurrence; or several such pairs), compiled in the module's namespace.  Tests install it with
pytest's monkeypatch, run a pin, and assert that the pin now fails.  Nothing
here changes the oracle's files.
"""
import inspect
import textwrap


def mutated(module, name, old, new=None):
    """old/new: one replacement, or old = a list of (old, new) pairs."""
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    pairs = old if new is None else [(old, new)]
    for a, b in pairs:
        n = src.count(a)
        if n != 1:
            raise AssertionError(f"{name}: expected one occurrence of {a!r}, found {n}")
        src = src.replace(a, b)
    ns = dict(vars(module))
    exec(compile(src, f"<mutated {module.__name__}.{name}>", "exec"), ns)
    return ns[name]
