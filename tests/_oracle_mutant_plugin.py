"""pytest plugin: run the oracle's pins against a copy of one oracle module
with one planted mistake (tests/test_oracle_mutations.py drives it).

Loaded with ``-p _oracle_mutant_plugin`` (tests/ and the repository root on
PYTHONPATH).  When the environment variable TR_ORACLE_MUTANT holds a JSON
object {"module": name, "old": text, "new": text}, the module
``oracle.<name>`` is re-executed from its source with the single occurrence
of ``old`` replaced by ``new``, and every reference to the original module
object (the ``oracle`` package attribute, ``sys.modules`` and the other
oracle modules' globals) is rebound to the mutant before any test module is
imported.  An empty ``old`` re-executes the source unchanged: the control
run that shows the swap itself breaks nothing.  Without the variable the
plugin does nothing.
"""

import json
import os
import sys
import types


def _install(spec):
    import oracle

    name = "oracle." + spec["module"]
    path = os.path.join(os.path.dirname(oracle.__file__), spec["module"] + ".py")
    with open(path) as f:
        src = f.read()
    old, new = spec["old"], spec["new"]
    if old:
        count = src.count(old)
        if count != 1:
            raise RuntimeError("mutation text occurs %d times in %s" % (count, path))
        src = src.replace(old, new)
    orig = sys.modules[name]
    mut = types.ModuleType(name)
    mut.__file__ = path
    mut.__package__ = "oracle"
    sys.modules[name] = mut
    exec(compile(src, path, "exec"), mut.__dict__)
    setattr(oracle, spec["module"], mut)
    for mod in list(sys.modules.values()):
        if getattr(mod, "__name__", "").startswith("oracle"):
            for key, val in list(vars(mod).items()):
                if val is orig:
                    setattr(mod, key, mut)


_SPEC = os.environ.get("TR_ORACLE_MUTANT")
if _SPEC:
    _install(json.loads(_SPEC))
