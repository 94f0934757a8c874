"""bench.py runs its GPU arm only on a GPU machine; this CPU check catches a
name that a function reads but that nothing defines (a local lost in an
edit), which would otherwise surface only there."""
import builtins
import os
import symtable

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _undefined(table, module_names, outer=frozenset()):
    bad = []
    local = {s.get_name() for s in table.get_symbols()
             if s.is_assigned() or s.is_parameter() or s.is_imported()}
    for sym in table.get_symbols():
        name = sym.get_name()
        if (sym.is_referenced() and sym.is_global() and name not in module_names
                and name not in outer and not hasattr(builtins, name)):
            bad.append((table.get_name(), name))
    for child in table.get_children():
        bad += _undefined(child, module_names, outer | local)
    return bad


def test_bench_functions_reference_only_defined_names():
    path = os.path.join(ROOT, "bench.py")
    st = symtable.symtable(open(path).read(), path, "exec")
    module_names = {s.get_name() for s in st.get_symbols()}
    assert _undefined(st, module_names) == []
