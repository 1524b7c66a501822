"""The C ABI's documentation: every function declared in include/*.h has its own comment
that cites the passage of the paper it implements (section, algorithm, equation, theorem,
table or example) or says that it has no counterpart in the paper, and every function that
returns an fp_status states its error behaviour."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CITE = re.compile(r"\bSecs?\. \d|\bAlgorithm\b|\bAlg\. |\bEq\. |\bTheorem\b|\bTable\b|\bExample\b|no counterpart")
ERRORS = re.compile(r"\bFP_E[A-Z]+\b|\bErrors?\b")


def declarations():
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        for m in re.finditer(r"\n(fp_status|void|const char\*)\s+(fp_\w+)\s*\(", src):
            before = src[:m.start()]
            end = before.rfind("*/")
            last_stmt = max(before.rfind(";"), before.rfind("{"), before.rfind("}"))
            comment = before[before.rfind("/*", 0, end):end] if end > last_stmt else ""
            yield fn, m.group(2), m.group(1), re.sub(r"\s*\n\s*\*?\s?", " ", comment)


def test_every_declaration_cites_its_passage_and_errors():
    decls = list(declarations())
    assert len(decls) >= 30
    missing = [name for _, name, _, c in decls if not CITE.search(c)]
    assert not missing, f"no citation or 'no counterpart' note: {missing}"
    silent = [name for _, name, ret, c in decls if ret == "fp_status" and not ERRORS.search(c)]
    assert not silent, f"no error behaviour stated: {silent}"
